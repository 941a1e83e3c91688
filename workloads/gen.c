/*
 * gen.c -- seeded synthetic relations for the signature join.
 *
 * This module holds no part of the join or signature arithmetic: it only makes
 * input bytes.  Every random choice is a pure function of (seed, stream tag,
 * row, position) through the SplitMix64 finaliser (Steele, Lea, Flood 2014),
 * so the same relation is produced on any machine and by any number of
 * threads.
 *
 * A relation is a packed byte arena (keys back to back, no padding between
 * keys), n+1 uint64 offsets (key i is arena[off[i] .. off[i+1])) and n uint32
 * ids.  The arena allocation is rounded up to a 16-byte multiple plus 16 bytes
 * of zero padding.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

typedef struct {
    uint64_t seed;
    uint64_t m, n;                 /* |R|, |S| */
    uint32_t r_len_lo, r_len_hi;   /* R key length, uniform inclusive */
    uint32_t s_len_lo, s_len_hi;   /* fresh S key length, uniform inclusive */
    int32_t alphabet;              /* 0 printable 0x20..0x7E, 1 ACGT, 2 alnum, 3 any byte, 4 XML-like text */
    double frac_copy;              /* S rows that are exact copies of an R key */
    double frac_near;              /* S rows that are near-duplicates of an R key */
    int32_t near_lo, near_hi;      /* changed byte positions of a near-duplicate */
    double zipf_s;                 /* 0: partner R row uniform; else Zipf(s) over R rows */
    double dup_frac;               /* distinct R keys that occur more than once */
    int32_t dup_lo, dup_hi;        /* total occurrences of such a key */
} gen_spec;

/* the random choices (SplitMix64-based words, Feistel bijection, letters, XML
   text, key lengths) are shared with the device generator */
#include "genrng.h"

#define mix64 gen_mix64
#define rnd gen_rnd
#define uniform gen_uniform
#define perm gen_perm
#define letter gen_letter

static double unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

static const char ACGT[4] = {'A', 'C', 'G', 'T'};

/* bytes of the key with identity (rel, ident), written to dst[0..len) */
static void key_bytes(const gen_spec* sp, uint64_t rel, uint64_t ident, uint8_t* dst, uint64_t len) {
    if (sp->alphabet == 4) { gen_xml_bytes(sp->seed, T_BYTE + 16 * rel, ident, dst, len); return; }
    for (uint64_t j = 0; j < len; j += 4) {
        uint64_t r = gen_group_word(sp->seed, rel, ident, j >> 2);
        for (int q = 0; q < 4 && j + q < len; q++) dst[j + q] = letter(sp->alphabet, (uint16_t)(r >> (16 * q)));
    }
}

static uint32_t key_len(const gen_spec* sp, uint64_t rel, uint64_t ident) {
    return rel ? gen_key_len(sp->seed, rel, ident, sp->s_len_lo, sp->s_len_hi)
               : gen_key_len(sp->seed, rel, ident, sp->r_len_lo, sp->r_len_hi);
}

/*
 * Plan: which key each row holds.
 *   r_ident[m]: identity of R row r's key (rows sharing an identity are duplicates)
 *   r_len[m]  : its length
 *   s_kind[n] : 0 fresh random key, 1 exact copy of an R key, 2 near-duplicate
 *   s_src[n]  : R row copied (kinds 1, 2) or -1
 *   s_len[n]  : its length
 *   r_mult[m] : number of R rows holding the same key as row r (ground truth)
 * Returns 0 on success.
 */
int gen_plan(const gen_spec* sp, uint64_t* r_ident, uint32_t* r_len, uint32_t* r_mult,
             uint8_t* s_kind, int64_t* s_src, uint32_t* s_len) {
    uint64_t m = sp->m, n = sp->n;
    /* R: list each distinct key's occurrences consecutively, then scatter the
       list over the rows with a seeded bijection */
    uint64_t* G = (uint64_t*)malloc(sizeof(uint64_t) * (m ? m : 1));
    uint32_t* Gc = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    if (!G || !Gc) { free(G); free(Gc); return 1; }
    uint64_t filled = 0;
    for (uint64_t d = 0; filled < m; d++) {
        uint64_t c = 1;
        if (sp->dup_frac > 0 && unit(rnd(sp->seed, T_DUP, d, 0)) < sp->dup_frac)
            c = uniform(rnd(sp->seed, T_DUP, d, 1), (uint64_t)sp->dup_lo, (uint64_t)sp->dup_hi);
        if (c > m - filled) c = m - filled;
        for (uint64_t t = 0; t < c; t++) { G[filled + t] = d; Gc[filled + t] = (uint32_t)c; }
        filled += c;
    }
    for (uint64_t r = 0; r < m; r++) {
        uint64_t g = perm(sp->seed, T_PERM_R, m, r);
        r_ident[r] = G[g];
        r_mult[r] = Gc[g];
        r_len[r] = key_len(sp, 0, r_ident[r]);
    }
    free(G); free(Gc);

    /* Zipf partner choice: cumulative weights over ranks 1..m */
    double* cdf = NULL;
    if (sp->zipf_s > 0 && m > 0) {
        cdf = (double*)malloc(sizeof(double) * m);
        if (!cdf) return 1;
        double acc = 0;
        for (uint64_t k = 0; k < m; k++) { acc += pow((double)(k + 1), -sp->zipf_s); cdf[k] = acc; }
    }
    uint64_t n_copy = (uint64_t)llround(sp->frac_copy * (double)n);
    uint64_t n_near = (uint64_t)llround(sp->frac_near * (double)n);
    if (n_copy + n_near > n) n_near = n - n_copy;
    for (uint64_t j = 0; j < n; j++) {
        uint64_t p = perm(sp->seed, T_PERM_S, n, j);
        int kind = (m == 0) ? 0 : (p < n_copy ? 1 : (p < n_copy + n_near ? 2 : 0));
        s_kind[j] = (uint8_t)kind;
        if (kind == 0) {
            s_src[j] = -1;
            s_len[j] = key_len(sp, 1, j);
        } else {
            uint64_t r;
            uint64_t u = rnd(sp->seed, T_PARTNER, j, 0);
            if (cdf) {
                double x = unit(u) * cdf[m - 1];
                uint64_t lo = 0, hi = m - 1;           /* first rank with cdf > x */
                while (lo < hi) { uint64_t mid = (lo + hi) / 2; if (cdf[mid] > x) hi = mid; else lo = mid + 1; }
                r = perm(sp->seed, T_PERM_Z, m, lo);
            } else {
                r = u % m;
            }
            s_src[j] = (int64_t)r;
            s_len[j] = r_len[r];
        }
    }
    free(cdf);
    return 0;
}

typedef struct {
    const gen_spec* sp;
    const uint64_t* r_ident; const uint64_t* offR; uint8_t* arenaR;
    const uint8_t* s_kind; const int64_t* s_src; const uint64_t* offS; uint8_t* arenaS;
    uint64_t lo, hi; int which;
} fill_job;

static void near_dup(const gen_spec* sp, uint64_t j, uint8_t* key, uint64_t len) {
    if (len == 0) return;
    uint64_t c = uniform(rnd(sp->seed, T_NEARC, j, 0), (uint64_t)sp->near_lo, (uint64_t)sp->near_hi);
    if (c > len) c = len;
    uint64_t chosen[64];
    if (c > 64) c = 64;
    uint64_t draws = 0;
    for (uint64_t t = 0; t < c; t++) {
        uint64_t pos;
        int again;
        do {   /* distinct positions */
            pos = rnd(sp->seed, T_NEARP, j, draws++) % len;
            again = 0;
            for (uint64_t q = 0; q < t; q++) if (chosen[q] == pos) again = 1;
        } while (again);
        chosen[t] = pos;
        uint8_t old = key[pos];
        uint64_t r = rnd(sp->seed, T_NEARL, j, t);
        if (sp->alphabet == 1) {
            int idx = 0;
            for (int a = 0; a < 4; a++) if ((uint8_t)ACGT[a] == old) idx = a;
            key[pos] = (uint8_t)ACGT[(idx + 1 + (int)(r % 3)) & 3];
        } else {
            uint8_t nb;
            do { nb = letter(sp->alphabet, (uint16_t)r); r = mix64(r); } while (nb == old);
            key[pos] = nb;
        }
    }
}

static void* fill_worker(void* arg) {
    fill_job* f = (fill_job*)arg;
    for (uint64_t i = f->lo; i < f->hi; i++) {
        if (f->which == 0) {
            uint64_t len = f->offR[i + 1] - f->offR[i];
            key_bytes(f->sp, 0, f->r_ident[i], f->arenaR + f->offR[i], len);
        } else {
            uint8_t* dst = f->arenaS + f->offS[i];
            uint64_t len = f->offS[i + 1] - f->offS[i];
            if (f->s_kind[i] == 0) {
                key_bytes(f->sp, 1, i, dst, len);
            } else {
                uint64_t r = (uint64_t)f->s_src[i];
                memcpy(dst, f->arenaR + f->offR[r], len);
                if (f->s_kind[i] == 2) near_dup(f->sp, i, dst, len);
            }
        }
    }
    return NULL;
}

static void run_fill(fill_job base, uint64_t count, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > count) nthreads = count ? (int)count : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    fill_job* jobs = (fill_job*)malloc(sizeof(fill_job) * nthreads);
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = base;
        jobs[t].lo = count * t / nthreads;
        jobs[t].hi = count * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, fill_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th); free(jobs);
}

void gen_fill_R(const gen_spec* sp, const uint64_t* r_ident, const uint64_t* offR, uint8_t* arenaR, int nthreads) {
    fill_job b;
    memset(&b, 0, sizeof(b));
    b.sp = sp; b.r_ident = r_ident; b.offR = offR; b.arenaR = arenaR; b.which = 0;
    run_fill(b, sp->m, nthreads);
}

void gen_fill_S(const gen_spec* sp, const uint8_t* s_kind, const int64_t* s_src, const uint64_t* offS,
                uint8_t* arenaS, const uint64_t* offR, const uint8_t* arenaR, int nthreads) {
    fill_job b;
    memset(&b, 0, sizeof(b));
    b.sp = sp; b.s_kind = s_kind; b.s_src = s_src; b.offS = offS; b.arenaS = arenaS;
    b.offR = offR; b.arenaR = (uint8_t*)arenaR; b.which = 1;
    run_fill(b, sp->n, nthreads);
}

/* bytes of one key identity, for tests of the generator itself */
void gen_key_bytes(const gen_spec* sp, uint64_t rel, uint64_t ident, uint8_t* dst, uint64_t len) {
    key_bytes(sp, rel, ident, dst, len);
}

uint64_t gen_perm_x(uint64_t seed, uint64_t tag, uint64_t n, uint64_t x) { return perm(seed, tag, n, x); }

/* S rows that copy an R key: llround(frac_copy * n), as gen_plan counts them */
uint64_t gen_n_copy(double frac_copy, uint64_t n) { return (uint64_t)llround(frac_copy * (double)n); }
