// gf16.cuh -- GF(2^16) arithmetic and the algebraic-signature inner loop for
// sm_103a.
//
// Signature (Section 3.1 of the paper): for a key of l 16-bit symbols p_i,
//     sig^k = sum_{i=0}^{l-1} p_i * x^(k*i)  in GF(2^16) = GF(2)[x] / P(x),
// P(x) = x^16 + x^12 + x^3 + x + 1, k = 1..4, sums are XOR.
//
// Evaluation here is Horner's rule over 16-byte chunks (8 symbols), run from
// the last chunk to the first, with delayed reduction: the accumulator of
// component k is kept as an unreduced GF(2) polynomial in a 32-bit register,
// shifted by 8k bits per chunk and reduced back to 16 bits only when it would
// overflow.  A reduction clears the bits above 16 with two byte-indexed table
// lookups (bits 16..23 and 24..31), each entry holding b*x^16 (or b*x^24)
// mod P together with b shifted into the cleared byte, so that one XOR both
// removes the high byte and adds its residue.  The tables live in shared
// memory, one copy per bank so that the 32 lanes of a warp never conflict.
#pragma once
#include <cstdint>

namespace algsig {

constexpr uint32_t kPoly = 0x1100Bu;   // x^16 + x^12 + x^3 + x + 1
constexpr uint32_t kOrder = 65535u;    // order of x (x is primitive for this P)

// Shared-memory reduction tables: 256 rows of 256 bytes.  Row b holds, for
// every lane l, the bits-16..23 entry of byte b at word 32*... see below:
//   byte offset 256*b + 4*l        : T16[b] = (b * x^16 mod P) ^ (b << 16)
//   byte offset 256*b + 128 + 4*l  : T24[b] = (b * x^24 mod P) ^ (b << 24)
// Each lane reads its own bank, so the 32 lanes of a warp never conflict, and
// the byte address of an entry is (b << 8) | (4*l [+128]): one PRMT builds it
// from the unreduced value and the lane's offset.
constexpr int kRedWords = 256 * 64;
constexpr int kRedBytes = kRedWords * 4;

__host__ __device__ __forceinline__ uint32_t gf_times_x(uint32_t a) {
  a <<= 1;
  return (a & 0x10000u) ? (a ^ kPoly) : a;
}

// Fill the reduction tables.  `tmp` is 512 words of scratch shared memory.
// Must be called by the whole block; ends with __syncthreads().
__device__ __forceinline__ void init_red_tables(uint32_t* red, uint32_t* tmp) {
  for (int e = threadIdx.x; e < 512; e += blockDim.x) {
    const int tbl = e >> 8;            // 0: bits 16..23, 1: bits 24..31
    const uint32_t b = (uint32_t)(e & 255);
    uint32_t v = b;
    const int steps = 16 + 8 * tbl;    // b * x^16 or b * x^24
    for (int i = 0; i < steps; i++) v = gf_times_x(v);
    tmp[e] = v ^ (b << (16 + 8 * tbl));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kRedWords; i += blockDim.x) {
    const int b = i >> 6, tbl = (i >> 5) & 1;
    red[i] = tmp[tbl * 256 + b];
  }
  __syncthreads();
}

__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

// bytes (b_sel << 8) | low byte of `base`: byte 0 from base, byte 1 from u's byte
// `sel` (2 or 3), bytes 2..3 zero (base < 256)
__device__ __forceinline__ uint32_t tab_index(uint32_t u, uint32_t base, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(u), "r"(base), "r"(sel));
  return r;
}

// Per-lane table cursors: the lane's two offsets (4*l and 4*l + 128), and
// the load of the word at byte offset idx of the tables.  RedCursor takes the
// tables' shared address at run time; RedCursorAt400 has it as the load's
// immediate offset (one add less per lookup), valid when the tables start the
// dynamic shared memory and that begins right after the 1 KB every block
// reserves (shared address 0x400; the host checks this once per device).
struct RedCursor {
  uint32_t tab;       // shared byte address of the tables
  uint32_t off16;     // 4*lane
  uint32_t off24;     // 4*lane + 128
  uint32_t k16, nk16, k256;
  __device__ __forceinline__ uint32_t load(uint32_t idx) const { return lds32(tab + idx); }
};
__device__ uint32_t g_k16 = 0x10000u;   // 2^16, read at run time so the compiler keeps multiplies by it
struct RedCursorAt400 {
  uint32_t off16;
  uint32_t off24;
  uint32_t k16, nk16, k256;
  __device__ __forceinline__ uint32_t load(uint32_t idx) const {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1+1024];" : "=r"(v) : "r"(idx));
    return v;
  }
};
constexpr uint32_t kTablesAt400 = 0x400u;

__device__ __forceinline__ RedCursor red_cursor(const uint32_t* red) {
  RedCursor c;
  c.tab = (uint32_t)__cvta_generic_to_shared(red);
  c.off16 = 4u * (threadIdx.x & 31u);
  c.off24 = c.off16 + 128u;
  c.k16 = *(volatile uint32_t*)&g_k16; c.nk16 = 0u - c.k16; c.k256 = c.k16 >> 8;
  return c;
}
__device__ __forceinline__ RedCursorAt400 red_cursor_at400() {
  RedCursorAt400 c;
  c.off16 = 4u * (threadIdx.x & 31u);
  c.off24 = c.off16 + 128u;
  c.k16 = *(volatile uint32_t*)&g_k16; c.nk16 = 0u - c.k16; c.k256 = c.k16 >> 8;
  return c;
}

// PRMT selectors: result byte0 = base byte0 (index 4), byte1 = u byte 2 or 3,
// bytes 2, 3 = base byte 1 (index 5, zero)
constexpr uint32_t kSel16 = 0x5524u;
constexpr uint32_t kSel24 = 0x5534u;

// 32-bit unreduced value -> 16-bit residue mod P
template <class Cursor>
__device__ __forceinline__ uint32_t red32(uint32_t u, const Cursor& c) {
  const uint32_t t16 = c.load(tab_index(u, c.off16, kSel16));
  const uint32_t t24 = c.load(tab_index(u, c.off24, kSel24));
  return u ^ t16 ^ t24;
}

// value < 2^24 -> 16-bit residue (only bits 16..23 to clear)
template <class Cursor>
__device__ __forceinline__ uint32_t red24(uint32_t u, const Cursor& c) {
  return u ^ c.load(tab_index(u, c.off16, kSel16));
}

// One Horner step over a 16-byte chunk: acc_k <- acc_k * x^(8k) + sum_j q_j x^(kj),
// where q_{2t} = low half of word t and q_{2t+1} = high half of word t.
// Accumulators enter and leave reduced (< 2^16).  NCOMP = 2 computes only
// components 1 and 2 (the paper's two-symbol signature); a3, a4 stay as given.
template <int NCOMP = 4, class Cursor>
__device__ __forceinline__ void horner_chunk(uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3,
                                             uint32_t& a1, uint32_t& a2, uint32_t& a3, uint32_t& a4,
                                             const Cursor& rc) {
  // halves on the FMA pipe: h = hi32(v * 2^16), l = v - h * 2^16
  const uint32_t h0 = __umulhi(v0, rc.k16), l0 = h0 * rc.nk16 + v0;
  const uint32_t h1 = __umulhi(v1, rc.k16), l1 = h1 * rc.nk16 + v1;
  const uint32_t h2 = __umulhi(v2, rc.k16), l2 = h2 * rc.nk16 + v2;
  const uint32_t h3 = __umulhi(v3, rc.k16), l3 = h3 * rc.nk16 + v3;
  uint32_t u;
  // k = 1: 8 symbols, growth 8 bits
  u = (a1 << 8) ^ l0 ^ (h0 << 1) ^ (l1 << 2) ^ (h1 << 3) ^ (l2 << 4) ^ (h2 << 5) ^ (l3 << 6) ^ (h3 << 7);
  a1 = red24(u, rc);
  // k = 2: 8 symbols, growth 16 bits
  u = (a2 << 16) ^ l0 ^ (h0 << 2) ^ (l1 << 4) ^ (h1 << 6) ^ (l2 << 8) ^ (h2 << 10) ^ (l3 << 12) ^ (h3 << 14);
  a2 = red32(u, rc);
  if constexpr (NCOMP == 2) return;
  // k = 3: two halves of 4 symbols, growth 12 bits each (upper half first)
  u = (a3 << 12) ^ l2 ^ (h2 << 3) ^ (l3 << 6) ^ (h3 << 9);
  a3 = red32(u, rc);
  u = (a3 << 12) ^ l0 ^ (h0 << 3) ^ (l1 << 6) ^ (h1 << 9);
  a3 = red32(u, rc);
  // k = 4: two halves of 4 symbols, growth 16 bits each
  u = (a4 << 16) ^ l2 ^ (h2 << 4) ^ (l3 << 8) ^ (h3 << 12);
  a4 = red32(u, rc);
  u = (a4 << 16) ^ l0 ^ (h0 << 4) ^ (l1 << 8) ^ (h1 << 12);
  a4 = red32(u, rc);
}

// Mask of bytes [b0, b1) of a 16-byte chunk, for its 32-bit word j.
__device__ __forceinline__ uint32_t byte_range_mask(int b0, int b1, int j) {
  int lo = b0 - 4 * j, hi = b1 - 4 * j;
  lo = lo < 0 ? 0 : (lo > 4 ? 4 : lo);
  hi = hi < 0 ? 0 : (hi > 4 ? 4 : hi);
  const uint32_t mhi = hi >= 4 ? 0xFFFFFFFFu : ((1u << (8 * hi)) - 1u);
  const uint32_t mlo = lo >= 4 ? 0xFFFFFFFFu : ((1u << (8 * lo)) - 1u);
  return mhi & ~mlo;
}

// Murmur3 64-bit finaliser: bucket hash of (signature, length).
__device__ __forceinline__ uint64_t fmix64(uint64_t h) {
  h ^= h >> 33;
  h *= 0xff51afd7ed558ccdull;
  h ^= h >> 33;
  h *= 0xc4ceb9fe1a85ec53ull;
  h ^= h >> 33;
  return h;
}

__device__ __forceinline__ uint64_t sig_hash(uint64_t sig, uint64_t len) {
  return fmix64(sig ^ (len * 0x9E3779B97F4A7C15ull));
}

}  // namespace algsig
