/*
 * CPU oracle for fingerprint-filtered approximate keyword matching
 * (Cislak and Grabowski, "Lightweight Fingerprints for Fast Approximate
 * Keyword Matching Using Bitwise Operations", arXiv 1711.08475).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  The library never calls it
 * and shares no code, header, table or constant with it.
 *
 * What it computes, with the passage each part follows:
 *   orc_ham / orc_lev      Hamming and Levenshtein distance, Sec. 1.  Hamming
 *                          is the number of mismatching positions and is
 *                          infinite (returned as -1) for unequal lengths
 *                          (Sec. 3.3, proof of Theorem 1).  Levenshtein is the
 *                          full Wagner-Fischer dynamic programme: no band, no
 *                          early exit.
 *   orc_match              Keyword (dictionary) matching, Sec. 1: for every
 *                          pattern P, the ascending list of indices i with
 *                          D(P, S_i) <= k.  Brute force over every pair.  With
 *                          prune=1 the Levenshtein loop skips pairs whose
 *                          lengths differ by more than k (Lev >= |n-m|); the
 *                          tests check that prune=1 and prune=0 agree.
 *   orc_fp_*               The four fingerprints of Sec. 3 / Sec. 3.2, from a
 *                          symbol->field map (Sec. 3.2: "a mapping c -> q").
 *                          count is a saturating count min(c, 2^b - 1) stored
 *                          either in plain binary (the paper's encoding) or
 *                          reflected-Gray coded (this project's encoding).
 *   orc_fd                 Fingerprint distance F_D, Sec. 3.3: Hamming weight
 *                          of the XOR, or for position fingerprints the number
 *                          of mismatching p-bit fields plus the Hamming weight
 *                          of the XOR of the trailing occurrence bits.
 *   orc_symbol_map         Common / rare / mixed symbol sets, Sec. 3, chosen
 *                          by occurrence counts over the collection.
 *   orc_fd_count_l1        Count fingerprints compared field by field: the sum
 *                          over fields of |c1 - c2| of the saturating counts in
 *                          the paper's binary code (the remark after Eq. 1 in
 *                          Sec. 3.3 that the Hamming weight under-counts count
 *                          differences: 3 (11) against 1 (01) differ by 2).
 *   orc_qgram_map          q-gram fingerprints (the future work of Sec. 5: the
 *   orc_fp_qgram           fingerprint of Sec. 3.2 over q-grams instead of
 *                          single symbols): the sigma most frequent q-grams of
 *                          the collection each own a bit, set iff the q-gram
 *                          occurs in the string.  One edit touches at most q
 *                          q-grams on each side, so F_D grows by at most 2q
 *                          per edit and D >= ceil(F_D / 2q) (the argument of
 *                          Theorem 1 with 2q in place of 2).
 *   orc_filter_match_fps   The Sec. 4 method on given fingerprints and a given
 *   orc_bound_violations_fps  distance (Hamming weight, or the count L1), with
 *                          the bound D >= ceil(F_D / 2q) (q = 1: Eq. 1).
 *   orc_filter_match       The paper's own method, Sec. 4: the query
 *                          fingerprint is built once, each eligible word is
 *                          rejected when ceil(F_D/2) > k (Eq. 1), otherwise it
 *                          is verified: Hamming by a character loop that stops
 *                          once more than k mismatches are seen, Levenshtein
 *                          by the 2k+1 diagonal strip with two rows (Sec. 4).
 *
 * Every function above is pinned by the CPU tests (worked example of Sec. 3.1,
 * the run/ran example of Sec. 3.3, exhaustive edit-ball enumeration, the
 * Eq. 1 invariant, brute-force cross checks).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#define ORC_HAM 0
#define ORC_LEV 1

#define ORC_OCC 0
#define ORC_OCCH 1
#define ORC_COUNT 2
#define ORC_POS 3

/* ------------------------------------------------------------------------ */
/* Distances (Sec. 1)                                                        */
/* ------------------------------------------------------------------------ */

int64_t orc_ham(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m)
{
    if (n != m)
        return -1; /* infinite */
    int64_t d = 0;
    for (int64_t i = 0; i < n; i++)
        if (a[i] != b[i])
            d++;
    return d;
}

static int64_t min3(int64_t x, int64_t y, int64_t z)
{
    int64_t r = x < y ? x : y;
    return r < z ? r : z;
}

/* Wagner-Fischer: D[i][j] over all 0<=i<=n, 0<=j<=m, kept as two rows. */
static int64_t lev_rows(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                        int64_t *prev, int64_t *cur)
{
    for (int64_t j = 0; j <= m; j++)
        prev[j] = j;
    for (int64_t i = 1; i <= n; i++) {
        cur[0] = i;
        for (int64_t j = 1; j <= m; j++) {
            int64_t sub = prev[j - 1] + (a[i - 1] != b[j - 1]);
            cur[j] = min3(prev[j] + 1, cur[j - 1] + 1, sub);
        }
        int64_t *t = prev;
        prev = cur;
        cur = t;
    }
    return prev[m];
}

int64_t orc_lev(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m)
{
    int64_t stack_buf[2 * 514];
    int64_t *buf = stack_buf;
    if (m > 512) {
        buf = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(m + 1));
        if (!buf)
            return -2;
    }
    int64_t d = lev_rows(a, n, b, m, buf, buf + m + 1);
    if (buf != stack_buf)
        free(buf);
    return d;
}

/* ------------------------------------------------------------------------ */
/* Fingerprints (Sec. 3, Sec. 3.2)                                           */
/* ------------------------------------------------------------------------ */

/* Occurrence: bit q is set iff some symbol mapped to q occurs in s. */
uint32_t orc_fp_occ(const uint8_t *s, int64_t n, const int8_t *map)
{
    uint32_t fp = 0;
    for (int64_t i = 0; i < n; i++) {
        int q = map[s[i]];
        if (q >= 0)
            fp |= (uint32_t)1 << q;
    }
    return fp;
}

/* Occurrence halved: the first half is s[0, floor(n/2)), the second half the
 * rest.  Field q occupies bits 2q (first half) and 2q+1 (second half). */
uint32_t orc_fp_occh(const uint8_t *s, int64_t n, const int8_t *map)
{
    uint32_t fp = 0;
    int64_t half = n / 2;
    for (int64_t i = 0; i < n; i++) {
        int q = map[s[i]];
        if (q >= 0)
            fp |= (uint32_t)1 << (2 * q + (i >= half ? 1 : 0));
    }
    return fp;
}

/* Count: field q holds min(#occurrences of the symbols mapped to q, 2^b - 1)
 * at bits [b*q, b*q + b), in binary (gray=0, the paper's encoding) or as the
 * reflected Gray code v ^ (v >> 1) of that value (gray=1). */
uint32_t orc_fp_count(const uint8_t *s, int64_t n, const int8_t *map, int b, int gray)
{
    int64_t cnt[32];
    memset(cnt, 0, sizeof cnt);
    for (int64_t i = 0; i < n; i++) {
        int q = map[s[i]];
        if (q >= 0)
            cnt[q]++;
    }
    uint32_t sat = ((uint32_t)1 << b) - 1;
    uint32_t fp = 0;
    for (int q = 0; q < 32 && q * b < 32; q++) {
        uint32_t v = cnt[q] < (int64_t)sat ? (uint32_t)cnt[q] : sat;
        if (gray)
            v = v ^ (v >> 1);
        fp |= v << (b * q);
    }
    return fp;
}

/* Position: for the position fields j = 0..n_pos-1, the 0-indexed first
 * position of a symbol mapped to j, saturated at 2^p - 1, which also stands
 * for "absent"; field j occupies bits [p*j, p*j + p).  Symbols mapped to
 * n_pos + t are occurrence symbols and set bit p*n_pos + t. */
uint32_t orc_fp_pos(const uint8_t *s, int64_t n, const int8_t *map, int p, int n_pos)
{
    uint32_t sat = ((uint32_t)1 << p) - 1;
    uint32_t fp = 0;
    for (int j = 0; j < n_pos; j++) {
        uint32_t v = sat;
        for (int64_t i = 0; i < n; i++) {
            if (map[s[i]] == j) {
                v = i < (int64_t)sat ? (uint32_t)i : sat;
                break;
            }
        }
        fp |= v << (p * j);
    }
    for (int64_t i = 0; i < n; i++) {
        int q = map[s[i]];
        if (q >= n_pos)
            fp |= (uint32_t)1 << (p * n_pos + (q - n_pos));
    }
    return fp;
}

uint32_t orc_fingerprint(const uint8_t *s, int64_t n, const int8_t *map, int type, int b, int p,
                         int n_pos, int gray)
{
    switch (type) {
    case ORC_OCC:
        return orc_fp_occ(s, n, map);
    case ORC_OCCH:
        return orc_fp_occh(s, n, map);
    case ORC_COUNT:
        return orc_fp_count(s, n, map, b, gray);
    case ORC_POS:
        return orc_fp_pos(s, n, map, p, n_pos);
    }
    return 0;
}

void orc_fingerprint_many(const uint8_t *chars, const int64_t *off, int64_t n_str, const int8_t *map,
                          int type, int b, int p, int n_pos, int gray, uint32_t *out)
{
    for (int64_t i = 0; i < n_str; i++)
        out[i] = orc_fingerprint(chars + off[i], off[i + 1] - off[i], map, type, b, p, n_pos, gray);
}

static int weight(uint32_t x)
{
    int c = 0;
    while (x) {
        c += (int)(x & 1u);
        x >>= 1;
    }
    return c;
}

/* F_D (Sec. 3.3).  occ / occh / count: Hamming weight of the XOR.  pos: the
 * number of p-bit fields that differ, plus the Hamming weight of the XOR of
 * the occurrence bits above the fields. */
int orc_fd(uint32_t a, uint32_t b, int type, int width, int p, int n_pos)
{
    uint32_t wmask = width >= 32 ? 0xFFFFFFFFu : (((uint32_t)1 << width) - 1);
    uint32_t x = (a ^ b) & wmask;
    if (type != ORC_POS)
        return weight(x);
    int f = 0;
    uint32_t fmask = ((uint32_t)1 << p) - 1;
    for (int j = 0; j < n_pos; j++)
        if ((x >> (p * j)) & fmask)
            f++;
    int top = p * n_pos;
    return f + (top < 32 ? weight(x >> top) : 0);
}

/* Count fingerprints in the paper's binary code (Sec. 3.2), compared by the
 * distance of the counts themselves: field q (bits [bits*q, bits*q + bits)
 * below width) holds a saturating count; the result is the sum over fields of
 * |count1 - count2|.  A substitution moves one count down and one up by at
 * most one each, an insertion or deletion one count by at most one, so this
 * sum grows by at most 2 per edit and Eq. 1 holds for it. */
int orc_fd_count_l1(uint32_t a, uint32_t b, int width, int bits)
{
    uint32_t fmask = ((uint32_t)1 << bits) - 1;
    int f = 0;
    for (int q = 0; (q + 1) * bits <= width; q++) {
        int ca = (int)((a >> (bits * q)) & fmask);
        int cb = (int)((b >> (bits * q)) & fmask);
        f += ca > cb ? ca - cb : cb - ca;
    }
    return f;
}

/* ------------------------------------------------------------------------ */
/* q-gram fingerprints (Sec. 5, future work)                                */
/* ------------------------------------------------------------------------ */

static uint32_t gram_code(const uint8_t *s, int q)
{
    uint32_t c = 0;
    for (int j = 0; j < q; j++)
        c = (c << 8) | s[j];
    return c;
}

/* The sigma most frequent q-grams (1 <= q <= 3) over all positions of all
 * strings, most frequent first, ties broken by the smaller q-gram in byte
 * order (the code with the first byte most significant); only q-grams that
 * occur are eligible.  Field f is the f-th q-gram: its q bytes are written to
 * grams_out[f*q .. f*q+q) and its count to counts_out[f] (if given).
 * Returns the number of fields used, or -1 (bad q, or no memory). */
int orc_qgram_map(const uint8_t *chars, const int64_t *off, int64_t n_str, int q, int sigma,
                  uint8_t *grams_out, int64_t *counts_out)
{
    if (q < 1 || q > 3 || sigma < 0)
        return -1;
    size_t ncodes = (size_t)1 << (8 * q);
    int64_t *cnt = (int64_t *)calloc(ncodes, sizeof(int64_t));
    if (!cnt)
        return -1;
    for (int64_t i = 0; i < n_str; i++) {
        int64_t n = off[i + 1] - off[i];
        for (int64_t j = 0; j + q <= n; j++)
            cnt[gram_code(chars + off[i] + j, q)]++;
    }
    int used = 0;
    while (used < sigma) {
        size_t best = 0;
        int64_t bc = 0;
        for (size_t c = 0; c < ncodes; c++)
            if (cnt[c] > bc) { /* strict: the first (smallest) code wins a tie */
                bc = cnt[c];
                best = c;
            }
        if (bc == 0)
            break;
        for (int j = 0; j < q; j++)
            grams_out[used * q + j] = (uint8_t)(best >> (8 * (q - 1 - j)));
        if (counts_out)
            counts_out[used] = bc;
        cnt[best] = 0; /* taken */
        used++;
    }
    free(cnt);
    return used;
}

/* Bit f is set iff the f-th q-gram of the map occurs somewhere in s. */
uint32_t orc_fp_qgram(const uint8_t *s, int64_t n, const uint8_t *grams, int n_grams, int q)
{
    uint32_t fp = 0;
    for (int64_t i = 0; i + q <= n; i++)
        for (int f = 0; f < n_grams && f < 32; f++)
            if (memcmp(s + i, grams + (size_t)f * q, (size_t)q) == 0)
                fp |= (uint32_t)1 << f;
    return fp;
}

void orc_fp_qgram_many(const uint8_t *chars, const int64_t *off, int64_t n_str, const uint8_t *grams,
                       int n_grams, int q, uint32_t *out)
{
    for (int64_t i = 0; i < n_str; i++)
        out[i] = orc_fp_qgram(chars + off[i], off[i + 1] - off[i], grams, n_grams, q);
}

/* ------------------------------------------------------------------------ */
/* Symbol sets (Sec. 3): common, rare, mixed                                */
/* ------------------------------------------------------------------------ */

#define ORC_SET_COMMON 0
#define ORC_SET_RARE 1
#define ORC_SET_MIXED 2

/* Symbols are ranked by their number of occurrences in the collection, ties
 * broken by the smaller byte value.  Only symbols that occur are eligible; if
 * fewer than sigma occur, the remaining fields stay unused.  Field numbers
 * follow the order of selection: common = most frequent first; rare = least
 * frequent first; mixed = ceil(sigma/2) most frequent (most frequent first)
 * followed by floor(sigma/2) least frequent of the rest (least frequent
 * first).  Every other byte maps to -1.  Returns the number of fields used. */
int orc_symbol_map(const uint8_t *chars, int64_t total, int set, int sigma, int8_t *map_out,
                   int64_t *counts_out)
{
    int64_t cnt[256];
    memset(cnt, 0, sizeof cnt);
    for (int64_t i = 0; i < total; i++)
        cnt[chars[i]]++;
    if (counts_out)
        memcpy(counts_out, cnt, sizeof cnt);
    int order[256], n_occ = 0;
    for (int c = 0; c < 256; c++)
        if (cnt[c] > 0)
            order[n_occ++] = c;
    /* insertion sort: descending count, then ascending byte */
    for (int i = 1; i < n_occ; i++) {
        int c = order[i], j = i - 1;
        while (j >= 0 && (cnt[order[j]] < cnt[c] || (cnt[order[j]] == cnt[c] && order[j] > c))) {
            order[j + 1] = order[j];
            j--;
        }
        order[j + 1] = c;
    }
    /* rare order: ascending count, then ascending byte */
    int rorder[256];
    for (int i = 0; i < n_occ; i++)
        rorder[i] = order[i];
    for (int i = 1; i < n_occ; i++) {
        int c = rorder[i], j = i - 1;
        while (j >= 0 && (cnt[rorder[j]] > cnt[c] || (cnt[rorder[j]] == cnt[c] && rorder[j] > c))) {
            rorder[j + 1] = rorder[j];
            j--;
        }
        rorder[j + 1] = c;
    }
    for (int c = 0; c < 256; c++)
        map_out[c] = -1;
    int used = 0;
    if (set == ORC_SET_COMMON) {
        for (int i = 0; i < n_occ && used < sigma; i++)
            map_out[order[i]] = (int8_t)used++;
    } else if (set == ORC_SET_RARE) {
        for (int i = 0; i < n_occ && used < sigma; i++)
            map_out[rorder[i]] = (int8_t)used++;
    } else {
        int n_common = (sigma + 1) / 2;
        for (int i = 0; i < n_occ && used < n_common; i++)
            map_out[order[i]] = (int8_t)used++;
        for (int i = 0; i < n_occ && used < sigma; i++)
            if (map_out[rorder[i]] < 0)
                map_out[rorder[i]] = (int8_t)used++;
    }
    return used;
}

/* ------------------------------------------------------------------------ */
/* The paper's verification routines (Sec. 4)                                */
/* ------------------------------------------------------------------------ */

/* Character loop that stops as soon as more than k mismatches are seen.
 * Returns 1 iff Ham(a, b) <= k. */
int orc_ham_within(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m, int k)
{
    if (n != m)
        return 0;
    int64_t e = 0;
    for (int64_t i = 0; i < n; i++)
        if (a[i] != b[i] && ++e > k)
            return 0;
    return 1;
}

/* Ukkonen's diagonal strip: only cells with |i - j| <= k are evaluated, cells
 * outside count as k+1, two rows are kept.  Returns 1 iff Lev(a, b) <= k. */
int orc_lev_within(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m, int k)
{
    int64_t d = n - m;
    if (d > k || -d > k)
        return 0;
    int64_t big = (int64_t)k + 1;
    int64_t stack_buf[2 * 514];
    int64_t *buf = stack_buf;
    if (m > 512) {
        buf = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(m + 1));
        if (!buf)
            return -2;
    }
    int64_t *prev = buf, *cur = buf + m + 1;
    for (int64_t j = 0; j <= m; j++)
        prev[j] = j <= k ? j : big;
    int result = 1;
    for (int64_t i = 1; i <= n; i++) {
        int64_t lo = i - k > 0 ? i - k : 0;
        int64_t hi = i + k < m ? i + k : m;
        int64_t row_min = big;
        /* the strip's neighbours just outside it read as k+1 */
        if (lo >= 1)
            cur[lo - 1] = big;
        if (hi + 1 <= m)
            cur[hi + 1] = big;
        for (int64_t j = lo; j <= hi; j++) {
            int64_t v;
            if (j == 0) {
                v = i;
            } else {
                int64_t sub = prev[j - 1] + (a[i - 1] != b[j - 1]);
                int64_t up = prev[j] + 1;
                int64_t left = cur[j - 1] + 1;
                v = min3(sub, up, left);
            }
            if (v > big)
                v = big;
            cur[j] = v;
            if (v < row_min)
                row_min = v;
        }
        if (row_min > k) {
            result = 0;
            break;
        }
        int64_t *t = prev;
        prev = cur;
        cur = t;
    }
    if (result)
        result = prev[m] <= k;
    if (buf != stack_buf)
        free(buf);
    return result;
}

/* ------------------------------------------------------------------------ */
/* Matchers: brute force, and the paper's filter + verify                    */
/* ------------------------------------------------------------------------ */

#define ORC_FD_WEIGHT 0   /* Hamming weight of the XOR (occurrence, q-gram) */
#define ORC_FD_COUNT_L1 1 /* orc_fd_count_l1 */

static int fd_given(uint32_t a, uint32_t b, int kind, int width, int bits)
{
    if (kind == ORC_FD_COUNT_L1)
        return orc_fd_count_l1(a, b, width, bits);
    return orc_fd(a, b, ORC_OCC, width, 0, 0);
}

typedef struct {
    int32_t *v;
    int64_t n, cap;
} ivec;

static int ivec_push(ivec *a, int32_t x)
{
    if (a->n == a->cap) {
        int64_t cap = a->cap ? 2 * a->cap : 8;
        int32_t *p = (int32_t *)realloc(a->v, sizeof(int32_t) * (size_t)cap);
        if (!p)
            return -1;
        a->v = p;
        a->cap = cap;
    }
    a->v[a->n++] = x;
    return 0;
}

typedef struct {
    /* inputs */
    const uint8_t *dchars;
    const int64_t *doff;
    int64_t nd;
    const uint8_t *qchars;
    const int64_t *qoff;
    int64_t nq;
    int k, metric, prune;
    /* filter mode */
    int use_filter, type, width, p, n_pos;
    int fd_kind, bits, qmul; /* given-fingerprint mode: distance kind, count bits, bound 2*qmul*k */
    const uint32_t *dfp;
    const uint32_t *qfp;
    /* outputs */
    ivec *rows;
    int64_t next;
    pthread_mutex_t mu;
    int64_t pairs, survivors;
    int failed;
} job_t;

static void run_query(job_t *J, int64_t q, int64_t *pairs, int64_t *surv, int64_t *prev, int64_t *cur)
{
    const uint8_t *P = J->qchars + J->qoff[q];
    int64_t n = J->qoff[q + 1] - J->qoff[q];
    ivec *row = &J->rows[q];
    for (int64_t i = 0; i < J->nd; i++) {
        const uint8_t *S = J->dchars + J->doff[i];
        int64_t m = J->doff[i + 1] - J->doff[i];
        int hit;
        if (J->use_filter) {
            /* eligible pairs: equal length (Ham) or |n - m| <= k (Lev) */
            if (J->metric == ORC_HAM ? (m != n) : (m - n > J->k || n - m > J->k))
                continue;
            (*pairs)++;
            if (J->use_filter == 1) {
                int f = orc_fd(J->qfp[q], J->dfp[i], J->type, J->width, J->p, J->n_pos);
                if ((f + 1) / 2 > J->k) /* Eq. 1: D >= ceil(F_D / 2) */
                    continue;
            } else {
                int f = fd_given(J->qfp[q], J->dfp[i], J->fd_kind, J->width, J->bits);
                int div = 2 * J->qmul;
                if ((f + div - 1) / div > J->k) /* D >= ceil(F_D / 2q) */
                    continue;
            }
            (*surv)++;
            hit = J->metric == ORC_HAM ? orc_ham_within(P, n, S, m, J->k)
                                       : orc_lev_within(P, n, S, m, J->k);
        } else if (J->metric == ORC_HAM) {
            int64_t d = orc_ham(P, n, S, m);
            hit = d >= 0 && d <= J->k;
        } else {
            if (J->prune && (m - n > J->k || n - m > J->k))
                continue;
            int64_t d = m + 1 > 513 ? orc_lev(P, n, S, m) : lev_rows(P, n, S, m, prev, cur);
            hit = d >= 0 && d <= J->k;
        }
        if (hit && ivec_push(row, (int32_t)i) != 0)
            J->failed = 1;
    }
}

static void *worker(void *arg)
{
    job_t *J = (job_t *)arg;
    int64_t prev[514], cur[514];
    int64_t pairs = 0, surv = 0;
    for (;;) {
        int64_t q = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (q >= J->nq)
            break;
        run_query(J, q, &pairs, &surv, prev, cur);
    }
    pthread_mutex_lock(&J->mu);
    J->pairs += pairs;
    J->survivors += surv;
    pthread_mutex_unlock(&J->mu);
    return NULL;
}

static int run_job(job_t *J, int nthreads, int64_t *row_ptr, int32_t **idx_out)
{
    J->rows = (ivec *)calloc((size_t)(J->nq > 0 ? J->nq : 1), sizeof(ivec));
    if (!J->rows)
        return -1;
    pthread_mutex_init(&J->mu, NULL);
    if (nthreads <= 0)
        nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 512)
        nthreads = 512;
    pthread_t th[512];
    int started = 0;
    for (int t = 1; t < nthreads; t++)
        if (pthread_create(&th[started], NULL, worker, J) == 0)
            started++;
    worker(J);
    for (int t = 0; t < started; t++)
        pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J->mu);
    int64_t total = 0;
    row_ptr[0] = 0;
    for (int64_t q = 0; q < J->nq; q++) {
        total += J->rows[q].n;
        row_ptr[q + 1] = total;
    }
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    if (!idx)
        J->failed = 1;
    for (int64_t q = 0; q < J->nq; q++) {
        if (idx && J->rows[q].n)
            memcpy(idx + row_ptr[q], J->rows[q].v, sizeof(int32_t) * (size_t)J->rows[q].n);
        free(J->rows[q].v);
    }
    free(J->rows);
    if (J->failed) {
        free(idx);
        return -1;
    }
    *idx_out = idx;
    return 0;
}

/* Brute-force keyword matching.  Rows come out in ascending dictionary order
 * because each query scans the dictionary from index 0 upwards.  *idx_out is
 * allocated here; release it with orc_free. */
int orc_match(const uint8_t *dchars, const int64_t *doff, int64_t nd, const uint8_t *qchars,
              const int64_t *qoff, int64_t nq, int k, int metric, int prune, int nthreads,
              int64_t *row_ptr, int32_t **idx_out)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.dchars = dchars;
    J.doff = doff;
    J.nd = nd;
    J.qchars = qchars;
    J.qoff = qoff;
    J.nq = nq;
    J.k = k;
    J.metric = metric;
    J.prune = prune;
    return run_job(&J, nthreads, row_ptr, idx_out);
}

/* The paper's method: fingerprints of the dictionary are built beforehand
 * (Sec. 3.4), the query fingerprint once per query (Sec. 4), each eligible
 * pair is rejected by Eq. 1 or verified.  stats[0] = eligible pairs,
 * stats[1] = pairs that passed the fingerprint test. */
int orc_filter_match(const uint8_t *dchars, const int64_t *doff, int64_t nd, const uint8_t *qchars,
                     const int64_t *qoff, int64_t nq, int k, int metric, int type, int width, int b,
                     int p, int gray, const int8_t *map, int nthreads, int64_t *row_ptr,
                     int32_t **idx_out, int64_t *stats)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.dchars = dchars;
    J.doff = doff;
    J.nd = nd;
    J.qchars = qchars;
    J.qoff = qoff;
    J.nq = nq;
    J.k = k;
    J.metric = metric;
    J.use_filter = 1;
    J.type = type;
    J.width = width;
    J.p = p;
    J.n_pos = type == ORC_POS ? width / p : 0;
    uint32_t *dfp = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nd > 0 ? nd : 1));
    uint32_t *qfp = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nq > 0 ? nq : 1));
    if (!dfp || !qfp) {
        free(dfp);
        free(qfp);
        return -1;
    }
    orc_fingerprint_many(dchars, doff, nd, map, type, b, p, J.n_pos, gray, dfp);
    orc_fingerprint_many(qchars, qoff, nq, map, type, b, p, J.n_pos, gray, qfp);
    J.dfp = dfp;
    J.qfp = qfp;
    int rc = run_job(&J, nthreads, row_ptr, idx_out);
    free(dfp);
    free(qfp);
    if (stats) {
        stats[0] = J.pairs;
        stats[1] = J.survivors;
    }
    return rc;
}

/* The Sec. 4 method on fingerprints computed by the caller: a pair is
 * rejected when ceil(F_D / 2q) > k, F_D of the given kind, otherwise
 * verified as in orc_filter_match.  q = 1 is Eq. 1. */
int orc_filter_match_fps(const uint8_t *dchars, const int64_t *doff, int64_t nd, const uint8_t *qchars,
                         const int64_t *qoff, int64_t nq, int k, int metric, const uint32_t *dfp,
                         const uint32_t *qfp, int fd_kind, int width, int bits, int q, int nthreads,
                         int64_t *row_ptr, int32_t **idx_out, int64_t *stats)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.dchars = dchars;
    J.doff = doff;
    J.nd = nd;
    J.qchars = qchars;
    J.qoff = qoff;
    J.nq = nq;
    J.k = k;
    J.metric = metric;
    J.use_filter = 2;
    J.fd_kind = fd_kind;
    J.width = width;
    J.bits = bits;
    J.qmul = q;
    J.dfp = dfp;
    J.qfp = qfp;
    int rc = run_job(&J, nthreads, row_ptr, idx_out);
    if (stats) {
        stats[0] = J.pairs;
        stats[1] = J.survivors;
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Exhaustive check of Eq. 1 (Theorems 1 and 2) over a set of strings        */
/* ------------------------------------------------------------------------ */

/* For every ordered pair (s, t) of the given strings with |len(s) - len(t)| <= 1
 * and a finite distance D (Ham needs equal lengths), count the pairs that
 * violate D(s, t) >= ceil(F_D(s', t') / 2).  out[0] = pairs examined,
 * out[1] = violations, out[2] = index of the first violating s (or -1),
 * out[3] = index of its t. */
void orc_bound_violations(const uint8_t *chars, const int64_t *off, int64_t n_str, const int8_t *map,
                          int type, int width, int b, int p, int gray, int metric, int64_t *out)
{
    int n_pos = type == ORC_POS ? width / p : 0;
    uint32_t *fp = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n_str > 0 ? n_str : 1));
    out[0] = out[1] = 0;
    out[2] = out[3] = -1;
    if (!fp)
        return;
    orc_fingerprint_many(chars, off, n_str, map, type, b, p, n_pos, gray, fp);
    for (int64_t i = 0; i < n_str; i++) {
        const uint8_t *s = chars + off[i];
        int64_t n = off[i + 1] - off[i];
        for (int64_t j = 0; j < n_str; j++) {
            const uint8_t *t = chars + off[j];
            int64_t m = off[j + 1] - off[j];
            if (m - n > 1 || n - m > 1)
                continue;
            int64_t d = metric == ORC_HAM ? orc_ham(s, n, t, m) : orc_lev(s, n, t, m);
            if (d < 0)
                continue;
            out[0]++;
            int f = orc_fd(fp[i], fp[j], type, width, p, n_pos);
            if (d < (f + 1) / 2) {
                if (out[1] == 0) {
                    out[2] = i;
                    out[3] = j;
                }
                out[1]++;
            }
        }
    }
    free(fp);
}

/* The same check on fingerprints computed by the caller, for the bound
 * D >= ceil(F_D / 2q) with F_D of the given kind (q = 1: Eq. 1). */
void orc_bound_violations_fps(const uint8_t *chars, const int64_t *off, int64_t n_str, const uint32_t *fp,
                              int fd_kind, int width, int bits, int q, int metric, int64_t *out)
{
    out[0] = out[1] = 0;
    out[2] = out[3] = -1;
    int div = 2 * q;
    for (int64_t i = 0; i < n_str; i++) {
        const uint8_t *s = chars + off[i];
        int64_t n = off[i + 1] - off[i];
        for (int64_t j = 0; j < n_str; j++) {
            const uint8_t *t = chars + off[j];
            int64_t m = off[j + 1] - off[j];
            if (m - n > 1 || n - m > 1)
                continue;
            int64_t d = metric == ORC_HAM ? orc_ham(s, n, t, m) : orc_lev(s, n, t, m);
            if (d < 0)
                continue;
            out[0]++;
            int f = fd_given(fp[i], fp[j], fd_kind, width, bits);
            if (d < (f + div - 1) / div) {
                if (out[1] == 0) {
                    out[2] = i;
                    out[3] = j;
                }
                out[1]++;
            }
        }
    }
}

void orc_free(void *p) { free(p); }
