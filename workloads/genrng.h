/*
 * genrng.h -- the counter-based random choices of the input generator, shared
 * by the host generator (gen.c, plain C) and the device generator (gen_dev.cu).
 *
 * Holds no part of the join or signature arithmetic.  Every choice is a pure
 * function of (seed, stream tag, a, b) through the SplitMix64 finaliser
 * (Steele, Lea, Flood 2014), so host and device produce the same bytes.
 * GEN_HD marks the functions for both sides (empty for a host compiler).
 */
#ifndef WORKLOADS_GENRNG_H
#define WORKLOADS_GENRNG_H

#include <stdint.h>

#ifndef GEN_HD
#define GEN_HD
#endif

/* stream tags */
enum { T_LEN = 1, T_BYTE, T_PERM_R, T_PERM_S, T_PERM_Z, T_PARTNER, T_DUP, T_NEARC, T_NEARP, T_NEARL };

GEN_HD static inline uint64_t gen_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* pure random 64-bit word for (seed, tag, a, b) */
GEN_HD static inline uint64_t gen_rnd(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b) {
    uint64_t h = gen_mix64(seed + 0x9E3779B97F4A7C15ull * (tag + 1));
    h = gen_mix64(h ^ (a * 0xD1B54A32D192ED03ull + 0x632BE59BD9B4E019ull));
    h = gen_mix64(h ^ (b * 0x8CB92BA72F3D8DD7ull + 0x2545F4914F6CDD1Dull));
    return h;
}

GEN_HD static inline uint64_t gen_uniform(uint64_t r, uint64_t lo, uint64_t hi) { /* inclusive */
    return lo + r % (hi - lo + 1);
}

/* bijection on [0, n): 4-round Feistel on the smallest even bit width that
   covers n, with cycle walking */
GEN_HD static inline uint64_t gen_perm(uint64_t seed, uint64_t tag, uint64_t n, uint64_t x) {
    if (n <= 1) return 0;
    int bits = 2;
    while (bits < 64 && (1ull << bits) < n) bits += 2;
    int half = bits / 2;
    uint64_t mask = (1ull << half) - 1;
    do {
        uint64_t L = x >> half, R = x & mask;
        for (int r = 0; r < 4; r++) {
            uint64_t F = gen_rnd(seed, tag, (uint64_t)r, R) & mask;
            uint64_t nL = R, nR = L ^ F;
            L = nL; R = nR;
        }
        x = (L << half) | R;
    } while (x >= n);
    return x;
}

/* alphabets: 0 printable 0x20..0x7E, 1 ACGT, 2 alnum, 3 any byte (4, XML-like
   text, is built from alnum letters and a..z tag names) */
GEN_HD static inline uint8_t gen_letter(int alphabet, uint16_t u) {
    switch (alphabet) {
        case 1: return (uint8_t)"ACGT"[u & 3];
        case 2: return (uint8_t)"0123456789ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz"[((uint32_t)u * 62u) >> 16];
        case 3: return (uint8_t)(u & 0xFF);
        default: return (uint8_t)(0x20 + (((uint32_t)u * 95u) >> 16));
    }
}

/* XML-like text: elements <t>text</t> with a tag t of 3..12 letters a..z and
   alphanumeric text of 1..64 characters, concatenated while they fit, then
   alphanumeric characters up to exactly len bytes */
GEN_HD static inline void gen_xml_bytes(uint64_t seed, uint64_t tagbase, uint64_t ident, uint8_t* dst, uint64_t len) {
    uint64_t pos = 0, ctr = 0;
    for (;;) {
        uint64_t r = gen_rnd(seed, tagbase, ident, ctr++);
        uint64_t tl = 3 + r % 10, cl = 1 + (r >> 8) % 64;
        uint64_t need = 2 * tl + cl + 5;   /* <t> text </t> */
        if (pos + need > len) break;
        uint8_t tagname[12];
        for (uint64_t i = 0; i < tl; i++) tagname[i] = (uint8_t)('a' + gen_rnd(seed, tagbase, ident, ctr++) % 26);
        dst[pos++] = '<';
        for (uint64_t i = 0; i < tl; i++) dst[pos++] = tagname[i];
        dst[pos++] = '>';
        for (uint64_t i = 0; i < cl; i++) dst[pos++] = gen_letter(2, (uint16_t)gen_rnd(seed, tagbase, ident, ctr++));
        dst[pos++] = '<';
        dst[pos++] = '/';
        for (uint64_t i = 0; i < tl; i++) dst[pos++] = tagname[i];
        dst[pos++] = '>';
    }
    while (pos < len) dst[pos++] = gen_letter(2, (uint16_t)gen_rnd(seed, tagbase, ident, ctr++));
}

/* the 4 bytes of group g (bytes 4g .. 4g+3) of the key with identity (rel,
   ident) for the letter alphabets 0..3 */
GEN_HD static inline uint64_t gen_group_word(uint64_t seed, uint64_t rel, uint64_t ident, uint64_t g) {
    return gen_rnd(seed, T_BYTE + 16 * rel, ident, g);
}

/* key length of identity (rel, ident): uniform in [lo, hi] */
GEN_HD static inline uint32_t gen_key_len(uint64_t seed, uint64_t rel, uint64_t ident, uint32_t lo, uint32_t hi) {
    return (uint32_t)gen_uniform(gen_rnd(seed, T_LEN + 16 * rel, ident, 0), lo, hi);
}

#endif
