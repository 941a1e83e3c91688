/*
 * oracle.c -- CPU oracle for the algebraic-signature equi-join.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path must compute.  Only tests/, the smoke check of
 * __graft_entry__ and the CPU-baseline / reference arm of bench.py may load
 * it.  It shares no code, header, table or constant generator with the CUDA
 * library: everything below is written from the paper's definitions.
 *
 * What it follows (Mokadem, Hameurlain, Morvan, "Equi join query acceleration
 * using algebraic signatures", IADIS 2008):
 *   - Section 3.1: symbols p_i (i = 0..l-1) are elements of GF(2^f); addition
 *     is XOR; multiplication uses logarithm / antilogarithm tables over a
 *     primitive element alpha; the n-symbol signature is the vector of
 *     sig^k(P) = sum_i p_i * alpha_k^i for a base (alpha_1..alpha_n).
 *   - Section 2: the simple hash join (build a hash table on the smaller
 *     relation R, probe it with every tuple of S, emit matching tuples) and
 *     the Grace hash join (partition both relations by the hash of the join
 *     attribute, then join each pair of partitions as in the simple join).
 *   - Figure 2: build on R, probe with S, materialise T.
 *
 * Readings taken where the paper is silent or garbled (each listed in the
 * design notes): f = 16, n = 4 components, alpha_k = x^k, field polynomial
 * x^16 + x^12 + x^3 + x + 1 (0x1100B), symbols are little-endian byte pairs
 * with an odd trailing byte taken as the low byte of a symbol whose high byte
 * is 0, summation index i = 0..l-1, packed signature word with component k in
 * bits [16(k-1), 16k).  The join result is the exact equi-join: every pair
 * (r.id, s.id) whose keys have the same length and the same bytes.
 *
 * Signature functions whose parity is pinned by the tests: or_gf_* (order of
 * x, agreement of two multiplication algorithms with a textbook polynomial
 * product), or_sig_* (special cases, linearity, concatenation, Vandermonde
 * distinctness), or_join_* (nested loop on tiny inputs, generator ground
 * truth).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define OR_POLY 0x1100Bu     /* x^16 + x^12 + x^3 + x + 1 */
#define OR_ORDER 65535u      /* 2^16 - 1: order of the multiplicative group */

/* ------------------------------------------------------------------ */
/* GF(2^16) arithmetic (Section 3.1)                                   */
/* ------------------------------------------------------------------ */

static uint16_t g_log[65536];
static uint16_t g_antilog[65535];
static int g_ready = 0;

/* Multiply by x and reduce by the field polynomial. */
static uint32_t times_x(uint32_t a) {
    a <<= 1;
    if (a & 0x10000u) a ^= OR_POLY;
    return a;
}

/* antilog[e] = x^e, log[x^e] = e, built by repeated multiplication by x.
 * log[0] is unused and left 0. Returns 0 if x does not generate all 65535
 * non-zero elements (i.e. if the polynomial were not primitive). */
int or_gf_init(void) {
    if (g_ready) return 1;
    uint32_t a = 1;
    for (uint32_t e = 0; e < OR_ORDER; e++) {
        g_antilog[e] = (uint16_t)a;
        g_log[a] = (uint16_t)e;
        a = times_x(a);
    }
    /* after 65535 steps we must be back at 1, and every non-zero element must
       have been visited exactly once */
    if (a != 1u) return 0;
    for (uint32_t v = 1; v < 65536u; v++)
        if (g_antilog[g_log[v]] != v) return 0;
    g_ready = 1;
    return 1;
}

void or_gf_tables(uint16_t* log_out, uint16_t* antilog_out) {
    or_gf_init();
    if (log_out) memcpy(log_out, g_log, sizeof(g_log));
    if (antilog_out) memcpy(antilog_out, g_antilog, sizeof(g_antilog));
}

/* Product through the log / antilog tables. */
uint16_t or_gf_mul_tab(uint16_t a, uint16_t b) {
    or_gf_init();
    if (a == 0 || b == 0) return 0;
    uint32_t e = (uint32_t)g_log[a] + (uint32_t)g_log[b];
    if (e >= OR_ORDER) e -= OR_ORDER;
    return g_antilog[e];
}

/* Product by shift-and-add: b * a = sum over set bits j of b of a * x^j. */
uint16_t or_gf_mul_shift(uint16_t a, uint16_t b) {
    uint32_t acc = 0, cur = a;
    for (int j = 0; j < 16; j++) {
        if ((b >> j) & 1u) acc ^= cur;
        cur = times_x(cur);
    }
    return (uint16_t)acc;
}

/* x^e for any e >= 0 (the element alpha^e with alpha = x). */
uint16_t or_gf_pow_x(uint64_t e) {
    or_gf_init();
    return g_antilog[e % OR_ORDER];
}

/* ------------------------------------------------------------------ */
/* Algebraic signatures (Section 3.1)                                  */
/* ------------------------------------------------------------------ */

/* symbol p_i of a key: bytes 2i (low) and 2i+1 (high); a missing high byte of
   an odd-length key is 0. */
static uint16_t symbol_at(const uint8_t* key, uint64_t len, uint64_t i) {
    uint16_t lo = key[2 * i];
    uint16_t hi = (2 * i + 1 < len) ? key[2 * i + 1] : 0;
    return (uint16_t)(lo | (hi << 8));
}

/* The definition: sig^k = XOR over i with p_i != 0 of antilog[(log p_i + k*i) mod 65535]. */
uint64_t or_sig_tables(const uint8_t* key, uint64_t len) {
    or_gf_init();
    uint64_t l = (len + 1) / 2;
    uint16_t s[4] = {0, 0, 0, 0};
    for (uint64_t i = 0; i < l; i++) {
        uint16_t p = symbol_at(key, len, i);
        if (p == 0) continue;
        uint64_t lp = g_log[p];
        for (int k = 1; k <= 4; k++) {
            uint64_t e = (lp + (uint64_t)k * (i % OR_ORDER)) % OR_ORDER;
            s[k - 1] ^= g_antilog[e];
        }
    }
    return (uint64_t)s[0] | ((uint64_t)s[1] << 16) | ((uint64_t)s[2] << 32) | ((uint64_t)s[3] << 48);
}

/* Independent route: Horner's rule from the last symbol down,
   s_k <- s_k * x^k + p_i, using the shift-and-add product only. */
uint64_t or_sig_horner(const uint8_t* key, uint64_t len) {
    uint64_t l = (len + 1) / 2;
    uint16_t s[4] = {0, 0, 0, 0};
    uint16_t xk[4];
    uint32_t a = 1;
    for (int k = 1; k <= 4; k++) { a = times_x(a); xk[k - 1] = (uint16_t)a; }  /* x^1..x^4 */
    for (uint64_t t = l; t > 0; t--) {
        uint16_t p = symbol_at(key, len, t - 1);
        for (int k = 0; k < 4; k++) s[k] = (uint16_t)(or_gf_mul_shift(s[k], xk[k]) ^ p);
    }
    return (uint64_t)s[0] | ((uint64_t)s[1] << 16) | ((uint64_t)s[2] << 32) | ((uint64_t)s[3] << 48);
}

typedef struct {
    const uint8_t* arena; const uint64_t* off; uint64_t lo, hi; uint64_t* out; int method;
} sig_job;

static void* sig_worker(void* arg) {
    sig_job* j = (sig_job*)arg;
    for (uint64_t i = j->lo; i < j->hi; i++) {
        const uint8_t* k = j->arena + j->off[i];
        uint64_t len = j->off[i + 1] - j->off[i];
        j->out[i] = j->method ? or_sig_horner(k, len) : or_sig_tables(k, len);
    }
    return NULL;
}

/* Signatures of n keys of a packed relation (arena + n+1 offsets).
   method 0 = table definition, 1 = Horner. */
void or_sig_batch(const uint8_t* arena, const uint64_t* off, uint64_t n, uint64_t* out, int method, int nthreads) {
    or_gf_init();
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > n) nthreads = n ? (int)n : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    sig_job* jobs = (sig_job*)malloc(sizeof(sig_job) * nthreads);
    for (int t = 0; t < nthreads; t++) {
        jobs[t].arena = arena; jobs[t].off = off; jobs[t].out = out; jobs[t].method = method;
        jobs[t].lo = n * t / nthreads; jobs[t].hi = n * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, sig_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th); free(jobs);
}

/* ------------------------------------------------------------------ */
/* Joins on full strings (Section 2, Figure 2)                         */
/* ------------------------------------------------------------------ */

static int key_equal(const uint8_t* a, uint64_t la, const uint8_t* b, uint64_t lb) {
    return la == lb && (la == 0 || memcmp(a, b, la) == 0);
}

static void emit(uint32_t* pairs, uint64_t cap, uint64_t* cnt, uint32_t r, uint32_t s) {
    if (*cnt < cap) { pairs[2 * *cnt] = r; pairs[2 * *cnt + 1] = s; }
    (*cnt)++;
}

static uint32_t id_of(const uint32_t* ids, uint64_t row) { return ids ? ids[row] : (uint32_t)row; }

/* Nested-loop join: every (r, s) pair is compared byte for byte. */
uint64_t or_join_nested(const uint8_t* aR, const uint64_t* oR, const uint32_t* idR, uint64_t m,
                        const uint8_t* aS, const uint64_t* oS, const uint32_t* idS, uint64_t n,
                        uint32_t* pairs, uint64_t cap) {
    uint64_t cnt = 0;
    for (uint64_t r = 0; r < m; r++)
        for (uint64_t s = 0; s < n; s++)
            if (key_equal(aR + oR[r], oR[r + 1] - oR[r], aS + oS[s], oS[s + 1] - oS[s]))
                emit(pairs, cap, &cnt, id_of(idR, r), id_of(idS, s));
    return cnt;
}

/* FNV-1a over the key bytes: the hash function h applied to the join attribute. */
static uint64_t str_hash(const uint8_t* p, uint64_t len) {
    uint64_t h = 1469598103934665603ull;
    for (uint64_t i = 0; i < len; i++) { h ^= p[i]; h *= 1099511628211ull; }
    h ^= len;
    h *= 0x9E3779B97F4A7C15ull;
    return h ^ (h >> 29);
}

/* Simple hash join restricted to rows rlist[0..m) of R and slist[0..n) of S:
   build: chained hash table (bucket headers + cell chains) on R's full keys;
   probe: every S key walks its bucket chain and is compared byte for byte. */
static uint64_t simple_join_rows(const uint8_t* aR, const uint64_t* oR, const uint32_t* idR,
                                 const uint64_t* rlist, uint64_t m,
                                 const uint8_t* aS, const uint64_t* oS, const uint32_t* idS,
                                 const uint64_t* slist, uint64_t n,
                                 uint32_t* pairs, uint64_t cap) {
    uint64_t nb = 1;
    while (nb < 2 * m) nb <<= 1;
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * nb);
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (m ? m : 1));
    uint64_t* hv = (uint64_t*)malloc(sizeof(uint64_t) * (m ? m : 1));
    for (uint64_t b = 0; b < nb; b++) head[b] = -1;
    for (uint64_t t = 0; t < m; t++) {
        uint64_t r = rlist ? rlist[t] : t;
        hv[t] = str_hash(aR + oR[r], oR[r + 1] - oR[r]);
        uint64_t b = hv[t] & (nb - 1);
        next[t] = head[b];
        head[b] = (int64_t)t;
    }
    uint64_t cnt = 0;
    for (uint64_t u = 0; u < n; u++) {
        uint64_t s = slist ? slist[u] : u;
        const uint8_t* ks = aS + oS[s];
        uint64_t ls = oS[s + 1] - oS[s];
        uint64_t h = str_hash(ks, ls);
        for (int64_t t = head[h & (nb - 1)]; t >= 0; t = next[t]) {
            uint64_t r = rlist ? rlist[t] : (uint64_t)t;
            if (hv[t] == h && key_equal(aR + oR[r], oR[r + 1] - oR[r], ks, ls))
                emit(pairs, cap, &cnt, id_of(idR, r), id_of(idS, s));
        }
    }
    free(head); free(next); free(hv);
    return cnt;
}

uint64_t or_join_simple(const uint8_t* aR, const uint64_t* oR, const uint32_t* idR, uint64_t m,
                        const uint8_t* aS, const uint64_t* oS, const uint32_t* idS, uint64_t n,
                        uint32_t* pairs, uint64_t cap) {
    return simple_join_rows(aR, oR, idR, NULL, m, aS, oS, idS, NULL, n, pairs, cap);
}

/* Grace hash join: partition R and S by the top bits of the key hash, then
   join each pair of partitions with the simple join, partitions spread over
   worker threads.  Each worker appends into its own growable buffer; the
   buffers are concatenated at the end. */
typedef struct {
    const uint8_t *aR, *aS; const uint64_t *oR, *oS; const uint32_t *idR, *idS;
    uint64_t** rpart; uint64_t* rcnt; uint64_t** spart; uint64_t* scnt;
    int nparts, first, step;
    uint32_t* out; uint64_t room; uint64_t cnt;
} grace_job;

static void* grace_worker(void* arg) {
    grace_job* g = (grace_job*)arg;
    g->cnt = 0;
    g->room = 1024;
    g->out = (uint32_t*)malloc(sizeof(uint32_t) * 2 * g->room);
    for (int p = g->first; p < g->nparts; p += g->step) {
        for (;;) {
            uint64_t left = g->room - g->cnt;
            uint64_t c = simple_join_rows(g->aR, g->oR, g->idR, g->rpart[p], g->rcnt[p],
                                          g->aS, g->oS, g->idS, g->spart[p], g->scnt[p],
                                          g->out + 2 * g->cnt, left);
            if (c <= left) { g->cnt += c; break; }
            /* not enough room: grow to fit this partition's exact count and redo it */
            while (g->room - g->cnt < c) g->room *= 2;
            g->out = (uint32_t*)realloc(g->out, sizeof(uint32_t) * 2 * g->room);
        }
    }
    return NULL;
}

static void partition_rows(const uint8_t* a, const uint64_t* o, uint64_t n, int nparts, int shift,
                           uint64_t*** part_out, uint64_t** cnt_out) {
    uint64_t* cnt = (uint64_t*)calloc(nparts, sizeof(uint64_t));
    uint32_t* pid = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    for (uint64_t i = 0; i < n; i++) {
        pid[i] = (uint32_t)(str_hash(a + o[i], o[i + 1] - o[i]) >> shift);
        cnt[pid[i]]++;
    }
    uint64_t** part = (uint64_t**)malloc(sizeof(uint64_t*) * nparts);
    uint64_t* fill = (uint64_t*)calloc(nparts, sizeof(uint64_t));
    for (int p = 0; p < nparts; p++) part[p] = (uint64_t*)malloc(sizeof(uint64_t) * (cnt[p] ? cnt[p] : 1));
    for (uint64_t i = 0; i < n; i++) part[pid[i]][fill[pid[i]]++] = i;
    free(fill); free(pid);
    *part_out = part; *cnt_out = cnt;
}

uint64_t or_join_grace(const uint8_t* aR, const uint64_t* oR, const uint32_t* idR, uint64_t m,
                       const uint8_t* aS, const uint64_t* oS, const uint32_t* idS, uint64_t n,
                       uint32_t* pairs, uint64_t cap, int log2_parts, int nthreads) {
    if (log2_parts < 1) log2_parts = 1;
    if (log2_parts > 16) log2_parts = 16;
    if (nthreads < 1) nthreads = 1;
    int nparts = 1 << log2_parts;
    int shift = 64 - log2_parts;
    uint64_t **rpart, **spart, *rcnt, *scnt;
    partition_rows(aR, oR, m, nparts, shift, &rpart, &rcnt);
    partition_rows(aS, oS, n, nparts, shift, &spart, &scnt);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    grace_job* jobs = (grace_job*)malloc(sizeof(grace_job) * nthreads);
    for (int t = 0; t < nthreads; t++) {
        grace_job* g = &jobs[t];
        g->aR = aR; g->aS = aS; g->oR = oR; g->oS = oS; g->idR = idR; g->idS = idS;
        g->rpart = rpart; g->rcnt = rcnt; g->spart = spart; g->scnt = scnt;
        g->nparts = nparts; g->first = t; g->step = nthreads;
        pthread_create(&th[t], NULL, grace_worker, g);
    }
    uint64_t total = 0;
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; t++) {
        for (uint64_t i = 0; i < jobs[t].cnt; i++) {
            if (total < cap) { pairs[2 * total] = jobs[t].out[2 * i]; pairs[2 * total + 1] = jobs[t].out[2 * i + 1]; }
            total++;
        }
        free(jobs[t].out);
    }
    for (int p = 0; p < nparts; p++) { free(rpart[p]); free(spart[p]); }
    free(rpart); free(spart); free(rcnt); free(scnt); free(th); free(jobs);
    return total;
}

/* ------------------------------------------------------------------ */
/* Byte symbols: GF(2^8) (Section 3.1: "a symbol is either a byte or a */
/* double byte")                                                       */
/* ------------------------------------------------------------------ */

/* Reading: field polynomial x^8 + x^4 + x^3 + x^2 + 1 (0x11D), alpha_k = x^k,
   symbol p_i = byte i, 4 components packed with component k in bits
   [8(k-1), 8k) of the low 32 bits. */
#define OR8_POLY 0x11Du
#define OR8_ORDER 255u

static uint8_t g8_log[256];
static uint8_t g8_antilog[255];
static int g8_ready = 0;

static uint32_t times_x8(uint32_t a) {
    a <<= 1;
    if (a & 0x100u) a ^= OR8_POLY;
    return a;
}

/* log / antilog of x by repeated multiplication; 1 if x is primitive */
int or_gf8_init(void) {
    if (g8_ready) return 1;
    uint32_t a = 1;
    for (uint32_t e = 0; e < OR8_ORDER; e++) {
        if (e > 0 && a == 1) return 0;
        g8_antilog[e] = (uint8_t)a;
        g8_log[a] = (uint8_t)e;
        a = times_x8(a);
    }
    if (a != 1) return 0;
    g8_ready = 1;
    return 1;
}

void or_gf8_tables(uint8_t* log_out, uint8_t* antilog_out) {
    or_gf8_init();
    if (log_out) memcpy(log_out, g8_log, sizeof(g8_log));
    if (antilog_out) memcpy(antilog_out, g8_antilog, sizeof(g8_antilog));
}

/* The definition: sig^k = XOR over i with b_i != 0 of antilog[(log b_i + k*i) mod 255]. */
uint64_t or_sig8_tables(const uint8_t* key, uint64_t len) {
    or_gf8_init();
    uint8_t s[4] = {0, 0, 0, 0};
    for (uint64_t i = 0; i < len; i++) {
        if (key[i] == 0) continue;
        const uint64_t lb = g8_log[key[i]];
        for (int k = 1; k <= 4; k++) s[k - 1] ^= g8_antilog[(lb + (uint64_t)k * (i % OR8_ORDER)) % OR8_ORDER];
    }
    return (uint64_t)s[0] | ((uint64_t)s[1] << 8) | ((uint64_t)s[2] << 16) | ((uint64_t)s[3] << 24);
}

/* Independent route: Horner's rule from the last byte down, s_k <- s_k * x^k + b_i,
   multiplying by x with the shift-and-reduce step only. */
uint64_t or_sig8_horner(const uint8_t* key, uint64_t len) {
    uint32_t s[4] = {0, 0, 0, 0};
    for (uint64_t t = len; t > 0; t--) {
        for (int k = 0; k < 4; k++) {
            uint32_t a = s[k];
            for (int r = 0; r <= k; r++) a = times_x8(a);
            s[k] = a ^ key[t - 1];
        }
    }
    return (uint64_t)s[0] | ((uint64_t)s[1] << 8) | ((uint64_t)s[2] << 16) | ((uint64_t)s[3] << 24);
}

typedef struct {
    const uint8_t* arena; const uint64_t* off; uint64_t lo, hi; uint64_t* out; int method;
} sig8_job;

static void* sig8_worker(void* arg) {
    sig8_job* j = (sig8_job*)arg;
    for (uint64_t i = j->lo; i < j->hi; i++) {
        const uint8_t* k = j->arena + j->off[i];
        uint64_t len = j->off[i + 1] - j->off[i];
        j->out[i] = j->method ? or_sig8_horner(k, len) : or_sig8_tables(k, len);
    }
    return NULL;
}

void or_sig8_batch(const uint8_t* arena, const uint64_t* off, uint64_t n, uint64_t* out, int method, int nthreads) {
    or_gf8_init();
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > n) nthreads = n ? (int)n : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    sig8_job* jobs = (sig8_job*)malloc(sizeof(sig8_job) * nthreads);
    for (int t = 0; t < nthreads; t++) {
        jobs[t].arena = arena; jobs[t].off = off; jobs[t].out = out; jobs[t].method = method;
        jobs[t].lo = n * t / nthreads; jobs[t].hi = n * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, sig8_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th); free(jobs);
}
