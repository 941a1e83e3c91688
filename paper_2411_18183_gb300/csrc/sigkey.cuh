// sigkey.cuh -- the signature kernel: one key per lane, keys grouped by
// length, components 1, 2 and 4 from a bit-sliced GF(2) Horner state.
//
// Arithmetic (Section 3.1: sig^k = sum_i p_i x^(k i), k = 1..4).  A key is
// read as 32-bit words v_t = p_{2t} | p_{2t+1} << 16 of its realigned stream
// (shifted by one byte when the key starts at an odd byte, so that symbols
// sit on 16-bit boundaries; word 0 starts at the key's first 32-byte block).
// Bit b of v_t is bit b of symbol 2t (b < 16) or bit b-16 of symbol 2t+1.
// For each of the 32 bit positions b ("planes") let
//     D_b(y) = sum_t bit_b(v_t) y^t,   a polynomial over GF(2).
// Then, with weights W_k(b) = x^b (b < 16) and x^(b - 16 + k) (b >= 16),
//     sig^k = sum_b W_k(b) D_b(x^(2k)).
// For k = 1, 2, 4 the exponent 2k is a power of two, and evaluating a GF(2)
// polynomial commutes with squaring (Frobenius): D_b(x^(2k)) = D_b(x)^(2k).
// So the 32 field elements S_b = D_b(x) determine components 1, 2 and 4.
// They are kept transposed ("bit-sliced"): register c_m holds, in bit b,
// coefficient m of S_b.  Horner's rule over the words, from the last to the
// first, S <- S * x + v_t, is then a fixed XOR network on the 16 registers
// (multiplication by x shifts the registers and folds c_15 back through
// x^16 = x^12 + x^3 + x + 1), 12 logic operations per 16 bytes for all 32
// planes at once.  At the end of the key,
//     sig^k = sum_m x^(2 k m) (lo16(c_m) + x^k hi16(c_m))   (mod P),
// since S_b^(2k) = sum_m c_m[b] x^(2 k m).  Component 3 (2k = 6 is not a power
// of two) has its own bit-sliced state over theta = x^1536, a Frobenius
// conjugate of x^3 (so D_b(x^6) is a fixed GF(2)-linear image of D_b(theta)),
// kept in a basis of GF(2^16) where its Horner step is 13 logic operations per
// 16 bytes; xs3_net.h (written by gen_xs3.py) holds that step and the map back
// to polynomial coordinates.
//
// Scheduling.  Each warp owns a range of keys with an equal share of the work
// (key bytes + a fixed cost per key) and walks it in windows of kLKWin keys.  A window's keys are sorted by length, and the warp
// computes them in groups of 32 consecutive sorted keys, one key per lane, so
// the lanes of a group have (nearly) the same amount of work.  A lane streams
// its key from global memory in 32-byte blocks (one 256-bit load per block,
// read-only path, no L1 allocation: every DRAM sector is fetched once), from
// the key's last block to its first, kLKDepth blocks ahead of the arithmetic
// in registers.  Lanes of a group whose keys are shorter start later, so all
// lanes reach their first block in the group's last iteration and finish the
// signatures together.  (Staging the keys through shared memory was measured
// slower: per-lane 16-byte copies fetch each 32-byte sector twice, and a TMA
// bulk copy per lane is serialised because its operands are warp-uniform.)
// In a batch the keys are the joins' row ranges back to back ("virtual
// rows"): the warps split them by work across the joins, and a window
// ends with its join's rows so that its keys are consecutive in the relation.
#pragma once
#include <cstdint>

#include "xs3_net.h"

namespace algsig {

#ifndef ALGSIG_LK_FINISH
#define ALGSIG_LK_FINISH __forceinline__
#endif
#ifndef ALGSIG_LK_LDQUAL
#define ALGSIG_LK_LDQUAL volatile
#endif
// Kernel shapes: warps per block (one block per SM) and 32-byte blocks in
// flight per key.  More warps hide more latency, more blocks in flight per key
// need more registers; the batch autotuner picks one per batch.  Shape 0 is
// the default of single relations.
struct LKShape {
  int warps, depth;
};
constexpr LKShape kLKShapes[] = {{24, 2}, {16, 2}, {32, 1}};
constexpr int kLKShapeCount = sizeof(kLKShapes) / sizeof(kLKShapes[0]);
#ifndef ALGSIG_LK_WIN
#define ALGSIG_LK_WIN 256
#endif
constexpr int kLKWin = ALGSIG_LK_WIN;                 // keys per sorting window (a power of two)
constexpr uint32_t kLKNoKey = 0xFFFFFFFFu;            // empty sorting entry
// relations of this many keys and more are split over the warps by work (a
// search in the offsets); smaller ones by key count, which saves the search's
// dependent loads where they would be a large share of the kernel's time
constexpr uint64_t kLKSearchFrom = 1ull << 19;
// A key's work in key-byte equivalents is its length + kLKKeyCost (the window
// sort, masks and finishing): fitted to the kernel's rates on keys of 32-128
// and 2048-8192 bytes, it gives the rate on 256-1024 bytes within 1 %.  The
// warps' shares are cut on it, so that a relation (or batch) that mixes short
// and long keys leaves no warp with far more keys than the others.
constexpr uint64_t kLKKeyCost = 140;
constexpr int kLKIdxBits = kLKWin == 256 ? 8 : (kLKWin == 128 ? 7 : (kLKWin == 64 ? 6 : 10));
static_assert((1 << kLKIdxBits) == kLKWin, "window sizes 64, 128, 256");
constexpr uint32_t kLKNbCap = (1u << (31 - kLKIdxBits)) - 1u;   // block counts above sort together

struct LKWarp {
  uint64_t woff[kLKWin + 2];       // offsets of the window's keys (woff[i] = off[wb + i]), i <= wn
  uint32_t order[kLKWin];          // window entries by block count: (block count << 8 | index)
  uint32_t hist[256];              // the counting sort's bins (block counts, 255 and up in the last)
};
static_assert(kLKWin >= 64 && kLKWin <= 256, "the window sort: up to 8 entries and 8 bins per lane");
constexpr size_t kSmemLKMasks = 1056;                 // 33 rows of 32 bytes
// (the blocks in flight of a shape live in registers: its depth takes no shared memory)
constexpr size_t lk_smem_bytes(int warps, int /*depth*/, size_t scratch_per_warp = 0) {
  return (size_t)kRedBytes + 1024 + kSmemLKMasks + (size_t)warps * (sizeof(LKWarp) + scratch_per_warp);
}
static_assert(lk_smem_bytes(32, 1) <= 232448, "lane-per-key signature kernel: shared memory");

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

// One 32-byte block of key bytes.
struct Blk {
  uint32_t w[8];
};

// 32 bytes at the 32-byte aligned address p, read-only path without L1
// allocation.
__device__ __forceinline__ Blk ld_blk(const uint8_t* p) {
  Blk b;
  asm ALGSIG_LK_LDQUAL("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                       : "=r"(b.w[0]), "=r"(b.w[1]), "=r"(b.w[2]), "=r"(b.w[3]), "=r"(b.w[4]), "=r"(b.w[5]),
                         "=r"(b.w[6]), "=r"(b.w[7])
                       : "l"(p));
  return b;
}
// The same with bytes outside [lim_lo, lim_hi) (the arena's readable range)
// not read and returned as zero; they never hold key bytes.  Only keys in the
// arena's first or last 32 bytes need it (lk_edge_key).
__device__ __forceinline__ Blk ld_blk_checked(const uint8_t* p, const uint8_t* lim_lo, const uint8_t* lim_hi) {
  if (p >= lim_lo && p + 32 <= lim_hi) return ld_blk(p);
  Blk b;
#pragma unroll
  for (int i = 0; i < 8; i++) b.w[i] = 0;
  if (p >= lim_lo && p + 16 <= lim_hi) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    b.w[0] = v.x; b.w[1] = v.y; b.w[2] = v.z; b.w[3] = v.w;
  }
  if (p + 16 >= lim_lo && p + 32 <= lim_hi) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p + 16));
    b.w[4] = v.x; b.w[5] = v.y; b.w[6] = v.z; b.w[7] = v.w;
  }
  return b;
}

// Bit-sliced Horner step over one 16-byte chunk (words v0..v3, v3 last in the
// key): S <- S x^4 + v3 x^3 + v2 x^2 + v1 x + v0, with x^16 = x^12 + x^3 + x + 1.
__device__ __forceinline__ void xs_chunk(uint32_t (&c)[16], uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3) {
  const uint32_t n0 = c[12] ^ v0;
  const uint32_t n1 = c[12] ^ c[13] ^ v1;
  const uint32_t n2 = c[13] ^ c[14] ^ v2;
  const uint32_t n3 = c[12] ^ c[14] ^ c[15] ^ v3;
  const uint32_t n4 = c[0] ^ c[13] ^ c[15];
  const uint32_t n5 = c[1] ^ c[14];
  const uint32_t n6 = c[2] ^ c[15];
  const uint32_t n12 = c[8] ^ c[12];
  const uint32_t n13 = c[9] ^ c[13];
  const uint32_t n14 = c[10] ^ c[14];
  const uint32_t n15 = c[11] ^ c[15];
  c[15] = n15; c[14] = n14; c[13] = n13; c[12] = n12;
  c[11] = c[7]; c[10] = c[6]; c[9] = c[5]; c[8] = c[4]; c[7] = c[3];
  c[6] = n6; c[5] = n5; c[4] = n4; c[3] = n3; c[2] = n2; c[1] = n1; c[0] = n0;
}

// Component K (1, 2 or 4) from the bit-sliced state:
//   sum_m x^(2 K m) (lo16(c_m) + x^K hi16(c_m)) mod P,
// by Horner over m with a 32-bit accumulator reduced every 8/K steps.
template <int K, class Cursor>
__device__ __forceinline__ uint32_t xs_component(const uint32_t (&c)[16], const Cursor& rc) {
  constexpr int kEvery = 8 / K;
  uint32_t acc = 0;
#pragma unroll
  for (int m = 15; m >= 0; --m) {
    acc = (acc << (2 * K)) ^ (c[m] & 0xFFFFu) ^ ((c[m] >> 16) << K);
    if ((16 - m) % kEvery == 0) acc = red32(acc, rc);
  }
  return acc;
}

// Component 3 from its bit-sliced state: with p_i = the poly coordinate i of
// every D_b(x^6) (bit b), sum_i x^i (lo16(p_i) + x^3 hi16(p_i)) mod P, by
// Horner over i with a 32-bit accumulator reduced once on the way.
template <class Cursor>
__device__ __forceinline__ uint32_t xs3_component(const uint32_t (&c3)[16], const Cursor& rc) {
  uint32_t p[16];
  xs3_to_poly(c3, p);
  uint32_t acc = 0;
#pragma unroll
  for (int i = 15; i >= 0; --i) {
    acc = (acc << 1) ^ (p[i] & 0xFFFFu) ^ ((p[i] >> 16) << 3);   // degree <= 18 + (15 - i)
    if (i == 3) acc = red32(acc, rc);
  }
  return red32(acc, rc);
}

// x^-m * v in GF(2^16) for 0 <= m <= 60; inv32: the multiply table of x^-32
template <class Cursor>
__device__ __forceinline__ uint32_t mul_xinv(const uint16_t* inv32, uint32_t v, uint32_t m, const Cursor& rc) {
  if (m >= 32) {
    v = mulc(inv32, v);
    m -= 32;
  }
  const uint32_t d = mulc(inv32, v);                     // v x^-32
  const uint64_t E = (uint64_t)d << (32 - m);            // v x^-32 x^(32-m), < 2^48
  const uint32_t r1 = red32((uint32_t)(E >> 16), rc);
  return red32(((uint32_t)E & 0xFFFFu) ^ (r1 << 16), rc);
}

// A lane's key in the current group.
struct LKKey {
  uint64_t kq;          // key index
  const uint8_t* base;  // 32-byte aligned address of the key's first block
  uint32_t nb;          // realigned 32-byte blocks (0: empty key)
  uint32_t a;           // offset of the key's first byte in its first block (0..31)
  uint32_t tail;        // bytes of the last aligned block that belong to the key, counted from its start
  bool valid;
  bool edge;            // a block of the key reaches outside the arena's readable range
};

// prefetch the offsets of the window starting at key wb (cp.async, one group)
__device__ __forceinline__ void lk_prefetch_window(LKWarp& W, const uint64_t* __restrict__ off, uint64_t wb,
                                                   uint64_t k_hi) {
  const uint32_t lane = threadIdx.x & 31u;
  if (wb < k_hi) {
    const uint64_t left = k_hi - wb;
    const uint32_t wn = left < (uint64_t)kLKWin ? (uint32_t)left : (uint32_t)kLKWin;
    for (uint32_t e = lane; e <= wn; e += 32) cp_async8(&W.woff[e], off + wb + e);
  }
  cp_async_commit();
}

// realigned 32-byte blocks of the key at absolute address abs
__device__ __forceinline__ uint32_t lk_blocks(uintptr_t abs, uint64_t len) {
  if (len == 0) return 0u;
  const uint64_t lo = (abs & 31u) & ~1ull;
  const uint64_t nb = (lo + len + 31) >> 5;
  return nb < 0xFFFFFFFFull ? (uint32_t)nb : 0xFFFFFFFFu;
}

// order the window's entries by block count: a counting sort over the block
// counts (255 and more share the last bin; the order within a bin is
// arbitrary), so that each group of 32 consecutive entries has keys of
// nearly equal length
__device__ __forceinline__ void lk_sort_window(LKWarp& W, uint32_t wn, uintptr_t arena) {
  const uint32_t lane = threadIdx.x & 31u;
  if (wn <= 32) {                                    // one group: nothing to balance
    for (uint32_t i = lane; i < (uint32_t)kLKWin; i += 32) W.order[i] = i < wn ? i : kLKNoKey;
    __syncwarp();
    return;
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) W.hist[8 * lane + t] = 0u;
  __syncwarp();
  constexpr int kPer = kLKWin / 32;                   // entries per lane
  uint32_t e[kPer], bin[kPer], rank[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const uint32_t i = lane + 32u * (uint32_t)j;
    e[j] = kLKNoKey;
    bin[j] = 0;
    rank[j] = 0;
    if (i < wn) {
      const uint64_t ks = W.woff[i], len = W.woff[i + 1] - ks;
      const uint32_t nb = lk_blocks(arena + ks, len);
      e[j] = ((nb < kLKNbCap ? nb : kLKNbCap) << kLKIdxBits) | i;
      bin[j] = nb < 255u ? nb : 255u;
      rank[j] = atomicAdd(&W.hist[bin[j]], 1u);
    }
  }
  __syncwarp();
  // exclusive prefix sum over the bins, 8 consecutive bins per lane
  uint32_t h[8], sum = 0;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    h[t] = W.hist[8 * lane + t];
    sum += h[t];
  }
  uint32_t incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(kFull, incl, d);
    if (lane >= (uint32_t)d) incl += o;
  }
  uint32_t base = incl - sum;
  __syncwarp();
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    W.hist[8 * lane + t] = base;
    base += h[t];
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < kPer; ++j)
    if (e[j] != kLKNoKey) W.order[W.hist[bin[j]] + rank[j]] = e[j];
  for (uint32_t i = wn + lane; i < (uint32_t)kLKWin; i += 32) W.order[i] = kLKNoKey;
  __syncwarp();
}

// group g of the window (wb: its first key) into the lanes; returns the
// group's iteration count (its longest key's blocks, at least 1)
__device__ __forceinline__ uint32_t lk_load_group(LKKey& k, const LKWarp& W, uint64_t wb, uint32_t g,
                                                  const uint8_t* arena, const uint8_t* lim_lo,
                                                  const uint8_t* lim_hi) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t e = W.order[32 * g + lane];
  k.valid = e != kLKNoKey;
  k.kq = 0; k.base = arena; k.nb = 0; k.a = 0; k.tail = 0; k.edge = false;
  if (k.valid) {
    const uint32_t i = e & (kLKWin - 1);
    const uint64_t ks = W.woff[i], len = W.woff[i + 1] - ks;
    const uintptr_t abs = reinterpret_cast<uintptr_t>(arena) + ks;
    k.kq = wb + i;
    k.base = reinterpret_cast<const uint8_t*>(abs & ~(uintptr_t)31);
    k.a = (uint32_t)(abs & 31u);
    k.nb = lk_blocks(abs, len);
    if (k.nb) k.tail = (uint32_t)((uint64_t)k.a + len - 32ull * (k.nb - 1));
    k.edge = k.nb && (k.base < lim_lo || k.base + 32ull * k.nb > lim_hi);
  }
  // an edge key is computed apart (lk_edge_key); the group's loop skips it
  const uint32_t G = __reduce_max_sync(kFull, k.edge ? 0u : k.nb);
  return G < 1u ? 1u : G;
}

// an empty slot (no key) for a lane
__device__ __forceinline__ uint32_t lk_no_group(LKKey& k, const uint8_t* arena) {
  k.valid = false;
  k.kq = 0; k.base = arena; k.nb = 0; k.a = 0; k.tail = 0; k.edge = false;
  return 1u;
}

// Byte masks of a 32-byte block in shared memory: row e (0..32) keeps bytes
// [0, e).  Masking a block is two 16-byte loads and eight logic operations.
constexpr int kLKMaskRows = 33;
__device__ __forceinline__ void lk_fill_masks(uint4* mt) {
  for (int i = threadIdx.x; i < kLKMaskRows * 2; i += blockDim.x) {
    const int e = i >> 1, h = i & 1;
    uint32_t m[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int r = e - 16 * h - 4 * j;
      m[j] = r <= 0 ? 0u : (r >= 4 ? ~0u : ((1u << (8 * r)) - 1u));
    }
    mt[i] = make_uint4(m[0], m[1], m[2], m[3]);
  }
}
// keep bytes [0, e) of a block (e >= 32 keeps all)
__device__ __forceinline__ void blk_keep_below(Blk& b, uint32_t e, const uint4* mt) {
  const uint32_t r = e < 32u ? e : 32u;
  const uint4 m0 = mt[2 * r], m1 = mt[2 * r + 1];
  b.w[0] &= m0.x; b.w[1] &= m0.y; b.w[2] &= m0.z; b.w[3] &= m0.w;
  b.w[4] &= m1.x; b.w[5] &= m1.y; b.w[6] &= m1.z; b.w[7] &= m1.w;
}
// zero bytes [0, a) of a block (a < 32)
__device__ __forceinline__ void blk_zero_below(Blk& b, uint32_t a, const uint4* mt) {
  const uint4 m0 = mt[2 * a], m1 = mt[2 * a + 1];
  b.w[0] &= ~m0.x; b.w[1] &= ~m0.y; b.w[2] &= ~m0.z; b.w[3] &= ~m0.w;
  b.w[4] &= ~m1.x; b.w[5] &= ~m1.y; b.w[6] &= ~m1.z; b.w[7] &= ~m1.w;
}

// the Horner steps of one 32-byte block (its two chunks, the upper one first)
template <int NCOMP, class Cursor>
__device__ __forceinline__ void lk_block(const Blk& w, uint32_t sh, uint32_t& nxt0, uint32_t (&c)[16],
                                         uint32_t (&c3)[16], const Cursor& rc) {
  uint32_t v[8];
#pragma unroll
  for (int i = 0; i < 7; i++) v[i] = __funnelshift_r(w.w[i], w.w[i + 1], sh);
  v[7] = __funnelshift_r(w.w[7], nxt0, sh);
  nxt0 = w.w[0];
  xs_chunk(c, v[4], v[5], v[6], v[7]);
  xs_chunk(c, v[0], v[1], v[2], v[3]);
  if constexpr (NCOMP == 4) {
    xs3_chunk(c3, v[4], v[5], v[6], v[7]);
    xs3_chunk(c3, v[0], v[1], v[2], v[3]);
  }
}

// A key's signature from the Horner state of its blocks (values counted from
// the first block's start; the key starts s = (a & ~1) / 2 symbols later).
template <int NCOMP, class Cursor>
__device__ ALGSIG_LK_FINISH uint64_t lk_finish(const uint32_t (&c)[16], const uint32_t (&c3)[16], uint32_t a,
                                              const uint16_t* inv32, const Cursor& rc) {
  const uint32_t v1 = xs_component<1>(c, rc);
  const uint32_t v2 = xs_component<2>(c, rc);
  const uint32_t s = (a & ~1u) >> 1;
  uint64_t sig = (uint64_t)mul_xinv(inv32, v1, s, rc) | ((uint64_t)mul_xinv(inv32, v2, 2 * s, rc) << 16);
  if constexpr (NCOMP == 4) {
    const uint32_t v3 = xs3_component(c3, rc);
    const uint32_t v4 = xs_component<4>(c, rc);
    sig |= ((uint64_t)mul_xinv(inv32, v3, 3 * s, rc) << 32) | ((uint64_t)mul_xinv(inv32, v4, 4 * s, rc) << 48);
  }
  return sig;
}

// The signature of a key with a block outside the arena's readable range
// (its first 32 bytes or its last): the blocks one by one with checked loads.
// At most a few keys per relation take this path.
// (one copy per kernel instantiation: ptxas fails on a non-inlined function
// shared by kernels of different shapes)
template <int NCOMP, int kLKWarps, int kLKDepth, bool BATCH, class Unique, class Cursor>
__device__ __noinline__ uint64_t lk_edge_key(const LKKey& k, const uint8_t* lim_lo, const uint8_t* lim_hi,
                                             const uint16_t* inv32, const uint4* mt, const Cursor& rc) {
  const uint32_t sh = 8u * (k.a & 1u);
  uint32_t nxt0 = 0;
  if (k.tail > 32u) nxt0 = __ldg(reinterpret_cast<const uint32_t*>(k.base + 32ull * k.nb));
  uint32_t c[16];
#pragma unroll
  for (int i = 0; i < 16; i++) c[i] = 0;
  uint32_t c3[16];                                    // component 3's state (unused with 2 components)
#pragma unroll
  for (int i = 0; i < 16; i++) c3[i] = 0;
  for (uint32_t vb = k.nb; vb-- > 0;) {
    Blk w = ld_blk_checked(k.base + 32ull * vb, lim_lo, lim_hi);
    if (vb + 1 == k.nb) blk_keep_below(w, k.tail, mt);
    if (vb == 0) blk_zero_below(w, k.a, mt);
    lk_block<NCOMP>(w, sh, nxt0, c, c3, rc);
  }
  return lk_finish<NCOMP>(c, c3, k.a, inv32, rc);
}

// The signatures of one group of keys: in iteration it of the group's G
// iterations the lane takes block vb = G - 1 - it of its key (its own blocks
// are vb < nb), so the lanes of shorter keys start later and every key reaches
// its block 0 in the group's last iteration.  An odd key whose last aligned
// block ends with a key byte needs the next block's first byte.  Keys with a
// block outside the arena's readable range are computed apart (lk_edge_key).
template <int NCOMP, int kLKWarps, int kLKDepth, bool BATCH, class Unique, class Cursor>
__device__ __forceinline__ uint64_t lk_group(const LKKey& k, uint32_t G, const uint8_t* lim_lo, const uint8_t* lim_hi,
                                         const uint16_t* inv32, const uint4* mt, uint64_t* __restrict__ sig_out,
                                         const Cursor& rc) {
  const uint32_t nb = k.edge ? 0u : k.nb;
  const uint32_t sh = 8u * (k.a & 1u);
  uint32_t nxt0 = 0;
  if (nb && k.tail > 32u) nxt0 = __ldg(reinterpret_cast<const uint32_t*>(k.base + 32ull * nb));
  // kLKDepth blocks in flight: iteration it takes its block out of ring slot it % kLKDepth and
  // refills the slot with block it + kLKDepth before computing (a ring of kLKDepth + 1 slots
  // written in place, and loads that run on into the next group, measured slower)
  Blk ring[kLKDepth];
#pragma unroll
  for (int u = 0; u < kLKDepth; ++u) {
#pragma unroll
    for (int i = 0; i < 8; i++) ring[u].w[i] = 0;
    const int vb = (int)G - 1 - u;
    if (vb >= 0 && (uint32_t)vb < nb) ring[u] = ld_blk(k.base + 32ull * (uint32_t)vb);
  }
  uint32_t c[16];
#pragma unroll
  for (int i = 0; i < 16; i++) c[i] = 0;
  uint32_t c3[16];                                    // component 3's state (unused with 2 components)
#pragma unroll
  for (int i = 0; i < 16; i++) c3[i] = 0;
  // all iterations but the last (block 0, the bytes before the key's start masked)
  const uint32_t M = G - 1;
  for (uint32_t it0 = 0; it0 < M; it0 += kLKDepth) {
#pragma unroll
    for (int u = 0; u < kLKDepth; ++u) {
      const uint32_t it = it0 + (uint32_t)u;
      if (it >= M) break;
      const uint32_t vb = G - 1 - it;
      Blk w = ring[u];
      if (it + kLKDepth < G) {
        const uint32_t vb2 = vb - kLKDepth;
        if (vb2 < nb) ring[u] = ld_blk(k.base + 32ull * vb2);
      }
      if (vb < nb) {
        if (vb + 1 == nb) blk_keep_below(w, k.tail, mt);   // bytes after the key's end
        lk_block<NCOMP>(w, sh, nxt0, c, c3, rc);
      }
    }
  }
  {                                                   // the last iteration: block 0 of every key
    static_assert(kLKDepth == 1 || kLKDepth == 2, "the last iteration's ring slot: depths 1 and 2");
    Blk w = ring[0];
    if constexpr (kLKDepth == 2) {
      if (M & 1u) w = ring[kLKDepth - 1];
    }
    if (nb) {
      if (nb == 1) blk_keep_below(w, k.tail, mt);
      blk_zero_below(w, k.a, mt);
      lk_block<NCOMP>(w, sh, nxt0, c, c3, rc);
    }
  }
  uint64_t sig = 0;
  if (k.valid && !k.edge) sig_out[k.kq] = sig = lk_finish<NCOMP>(c, c3, k.a, inv32, rc);
  if (__any_sync(kFull, k.edge))
    if (k.edge) sig_out[k.kq] = sig = lk_edge_key<NCOMP, kLKWarps, kLKDepth, BATCH, Unique>(k, lim_lo, lim_hi, inv32, mt, rc);
  return sig;
}

// What a kernel does with each group's signatures besides writing them out:
// nothing (LKNoPost), or a probe of a hash table (the whole join's fused
// pass).  kScratch: shared-memory bytes a warp needs for it.
struct LKNoPost {
  static constexpr size_t kScratch = 0;
  __device__ __forceinline__ void init(uint8_t*, const uint4*) {}
  __device__ __forceinline__ void group(uint64_t, uint64_t, bool) {}
  __device__ __forceinline__ void finish() {}
};

// The window of keys starting at key wb (keys below k_hi): returns its key
// count and sets *wa to its first row in the relation.  In a batch the keys are
// virtual rows (the joins' row ranges back to back) and a window ends with its
// join's rows, so that its keys are consecutive rows of the relation.
template <bool BATCH>
__device__ __forceinline__ uint32_t lk_window(const BatchJoin* __restrict__ J, int nj, int s_side, uint64_t wb,
                                              uint64_t k_hi, uint64_t* wa) {
  uint64_t lim = k_hi;
  *wa = wb;
  if constexpr (BATCH) {
    const int j = s_side ? join_of_virtual<true>(J, nj, wb) : join_of_virtual<false>(J, nj, wb);
    const uint64_t b = s_side ? __ldg(&J[j].s_begin) : __ldg(&J[j].r_begin);
    const uint64_t e = s_side ? __ldg(&J[j].s_end) : __ldg(&J[j].r_end);
    const uint64_t v0 = s_side ? __ldg(&J[j].vs) : __ldg(&J[j].vr);
    *wa = b + (wb - v0);
    if (v0 + (e - b) < lim) lim = v0 + (e - b);
  }
  const uint64_t left = lim - wb;
  return left < (uint64_t)kLKWin ? (uint32_t)left : (uint32_t)kLKWin;
}

// A warp's keys [lo, hi) of n (virtual rows of a batch side, or rows of a
// relation): equal counts below kLKSearchFrom keys, else equal shares of the
// work, key bytes + kLKKeyCost per key (in a batch, over the joins' keys back
// to back).  Whole warp.
template <bool BATCH>
__device__ __forceinline__ void lk_warp_range(const BatchJoin* __restrict__ J, int nj, int s_side,
                                              const uint64_t* __restrict__ off, uint64_t n, uint64_t warp,
                                              uint64_t nwarps, uint64_t* lo, uint64_t* hi) {
  if (n < kLKSearchFrom) {
    *lo = (uint64_t)((unsigned __int128)n * warp / nwarps);
    *hi = (uint64_t)((unsigned __int128)n * (warp + 1) / nwarps);
    return;
  }
  if constexpr (!BATCH) {
    warp_key_range(off, n, warp, nwarps, lo, hi, kLKKeyCost);
  } else {
    const uint64_t total = s_side ? vcost_of_join<true>(J, nj, kLKKeyCost) : vcost_of_join<false>(J, nj, kLKKeyCost);
    auto cut = [&](uint64_t w) -> uint64_t {
      if (w == 0) return 0;
      if (w >= nwarps) return n;
      const uint64_t t = (uint64_t)((unsigned __int128)total * w / nwarps);
      if (t >= total) return n;
      return s_side ? vcut_in_join<true>(J, off, join_of_vcost<true>(J, nj, t, kLKKeyCost), t, kLKKeyCost)
                    : vcut_in_join<false>(J, off, join_of_vcost<false>(J, nj, t, kLKKeyCost), t, kLKKeyCost);
    };
    *lo = cut(warp);
    *hi = cut(warp + 1);
  }
}

// The signatures of n keys: the rows of a relation (BATCH false), or the
// virtual rows of one side of a batch (BATCH true; s_side picks S, J and nj
// describe the joins, and sig_out is indexed by virtual row).
template <bool AT400, int NCOMP, int kLKWarps, int kLKDepth, bool BATCH, class Post = LKNoPost>
__global__ void __launch_bounds__(32 * kLKWarps, 1) sig_key_kernel(const uint8_t* __restrict__ arena,
                                                                const uint64_t* __restrict__ off, uint64_t n,
                                                                uint64_t* __restrict__ sig_out,
                                                                const BatchJoin* __restrict__ J, int nj, int s_side,
                                                                Post post = Post()) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* red = reinterpret_cast<uint32_t*>(smem);
  uint16_t* inv32 = reinterpret_cast<uint16_t*>(smem + kRedBytes);
  uint4* mt = reinterpret_cast<uint4*>(smem + kRedBytes + 1024);
  LKWarp* warps = reinterpret_cast<LKWarp*>(smem + kRedBytes + 1024 + kSmemLKMasks);
  post.init(smem + kRedBytes + 1024 + kSmemLKMasks + kLKWarps * sizeof(LKWarp) + (threadIdx.x >> 5) * Post::kScratch,
            reinterpret_cast<const uint4*>(smem + kRedBytes + 1024));
  lk_fill_masks(mt);
  for (int i = threadIdx.x; i < 256; i += blockDim.x)   // the x^-32 multiply table (512 entries)
    reinterpret_cast<uint32_t*>(inv32)[i] = reinterpret_cast<const uint32_t*>(g_const + 16 * 512)[i];
  const int wib = threadIdx.x >> 5;
  LKWarp& W = warps[wib];
  // the warp's keys and its first window's offsets first, so that their loads overlap the tables' copy
  const uint64_t warp = (uint64_t)blockIdx.x * kLKWarps + wib;
  const uint64_t nwarps = (uint64_t)gridDim.x * kLKWarps;
  uint64_t k_lo, k_hi;
  lk_warp_range<BATCH>(J, nj, s_side, off, n, warp, nwarps, &k_lo, &k_hi);
  uint64_t wa = 0;                                  // the current window: first row and key count
  uint32_t wn = k_lo < k_hi ? lk_window<BATCH>(J, nj, s_side, k_lo, k_hi, &wa) : 0u;
  if (wn) lk_prefetch_window(W, off, wa, wa + wn);
  // readable bytes of the arena: from its start to the 16-byte boundary after the relation's last key byte
  uint64_t rows_all = n;
  if constexpr (BATCH) rows_all = s_side ? __ldg(&J[nj].s_end) : __ldg(&J[nj].r_end);
  const uint8_t* lim_lo = arena;
  const uint8_t* lim_hi = arena + ((__ldg(off + rows_all) + 15) & ~15ull);
  for (int i = threadIdx.x; i < kRedWords / 4; i += blockDim.x)   // the reduction tables, from their image
    reinterpret_cast<uint4*>(red)[i] = g_red_img[i];
  __syncthreads();
  if (k_lo >= k_hi) return;
  using Cursor = typename std::conditional<AT400, RedCursorAt400, RedCursor>::type;
  Cursor rc;
  if constexpr (AT400) rc = red_cursor_at400(); else rc = red_cursor(red);

  for (uint64_t wb = k_lo; wb < k_hi;) {
    wn = lk_window<BATCH>(J, nj, s_side, wb, k_hi, &wa);   // as prefetched
    cp_async_wait_all();                            // the window's offsets
    __syncwarp();
    lk_sort_window(W, wn, reinterpret_cast<uintptr_t>(arena));
    const uint32_t ng = (wn + 31) / 32;
    for (uint32_t g = 0; g < ng; ++g) {
      LKKey k;
      const uint32_t G = lk_load_group(k, W, wb, g, arena, lim_lo, lim_hi);
      if (g + 1 == ng) {                            // the window's offsets are free: fetch the next ones
        __syncwarp();
        if (wb + wn < k_hi) {
          uint64_t na;
          const uint32_t nn = lk_window<BATCH>(J, nj, s_side, wb + wn, k_hi, &na);
          lk_prefetch_window(W, off, na, na + nn);
        }
      }
      const uint64_t sig = lk_group<NCOMP, kLKWarps, kLKDepth, BATCH, Post>(k, G, lim_lo, lim_hi, inv32, mt, sig_out, rc);
      post.group(k.kq, sig, k.valid);
    }
    wb += wn;
  }
  post.finish();
  cp_async_wait_all();
}

}  // namespace algsig
