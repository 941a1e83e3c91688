// gf8.cuh -- signatures with byte symbols over GF(2^8) (Section 3.1: a symbol
// is a byte or a double byte).  Field polynomial x^8 + x^4 + x^3 + x^2 + 1,
// alpha_k = x^k (k = 1..4), symbol p_i = byte i:
//     sig8^k = sum_{i=0}^{l-1} b_i x^(k i),   component k in bits [8(k-1), 8k).
//
// One thread per key runs Horner's rule from the key's last byte down,
// acc_k <- acc_k x^k + b_i.  Whole 16-byte chunks go four bytes at a time:
//     acc_k <- acc_k x^(4k) + b_(i+3) x^(3k) + b_(i+2) x^(2k) + b_(i+1) x^k + b_i,
// an unreduced GF(2) polynomial of at most 8 + 4k bits, folded back to 8 bits
// by byte-indexed table lookups (bits 8..15 and 16..23) whose entries also
// cancel the folded byte, as in gf16.cuh; the partial chunks at a key's ends
// go byte by byte.  The tables sit in shared memory, one copy per bank.
#pragma once
#include <cstdint>

#include "gf16.cuh"

namespace algsig {

constexpr uint32_t kPoly8 = 0x11Du;
constexpr int kG8Threads = 256;

__host__ __device__ __forceinline__ uint32_t gf8_times_x(uint32_t a) {
  a <<= 1;
  return (a & 0x100u) ? (a ^ kPoly8) : a;
}

// Fill the reduction tables (kRedWords words, the layout of gf16.cuh):
//   byte offset 256*b + 4*l        : b * x^8 mod P8 ^ (b << 8)    (folds bits 8..15)
//   byte offset 256*b + 128 + 4*l  : b * x^16 mod P8 ^ (b << 16)  (folds bits 16..23)
__device__ __forceinline__ void init_red8_tables(uint32_t* red, uint32_t* tmp) {
  for (int e = threadIdx.x; e < 512; e += blockDim.x) {
    const int tbl = e >> 8;
    const uint32_t b = (uint32_t)(e & 255);
    uint32_t v = b;
    for (int i = 0; i < 8 + 8 * tbl; i++) v = gf8_times_x(v);
    tmp[e] = v ^ (b << (8 + 8 * tbl));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kRedWords; i += blockDim.x) {
    const int b = i >> 6, tbl = (i >> 5) & 1;
    red[i] = tmp[tbl * 256 + b];
  }
  __syncthreads();
}

// PRMT selectors: byte 1 or byte 2 of u into the index's byte 1
constexpr uint32_t kSel8 = 0x5514u;
constexpr uint32_t kSel16b = 0x5524u;

// u < 2^24 -> residue mod P8 (< 256)
__device__ __forceinline__ uint32_t red8_24(uint32_t u, const RedCursor& c) {
  return u ^ c.load(tab_index(u, c.off16, kSel8)) ^ c.load(tab_index(u, c.off24, kSel16b));
}
// u < 2^16 -> residue mod P8
__device__ __forceinline__ uint32_t red8_16(uint32_t u, const RedCursor& c) {
  return u ^ c.load(tab_index(u, c.off16, kSel8));
}

// four bytes (b0 lowest address) into the four accumulators
__device__ __forceinline__ void gf8_word(uint32_t w, uint32_t& a1, uint32_t& a2, uint32_t& a3, uint32_t& a4,
                                         const RedCursor& rc) {
  const uint32_t b0 = w & 0xFFu, b1 = (w >> 8) & 0xFFu, b2 = (w >> 16) & 0xFFu, b3 = w >> 24;
  a1 = red8_16((a1 << 4) ^ (b3 << 3) ^ (b2 << 2) ^ (b1 << 1) ^ b0, rc);
  a2 = red8_16((a2 << 8) ^ (b3 << 6) ^ (b2 << 4) ^ (b1 << 2) ^ b0, rc);
  a3 = red8_24((a3 << 12) ^ (b3 << 9) ^ (b2 << 6) ^ (b1 << 3) ^ b0, rc);
  a4 = red8_24((a4 << 16) ^ (b3 << 12) ^ (b2 << 8) ^ (b1 << 4) ^ b0, rc);
}

// one byte
__device__ __forceinline__ void gf8_byte(uint32_t b, uint32_t& a1, uint32_t& a2, uint32_t& a3, uint32_t& a4,
                                         const RedCursor& rc) {
  a1 = red8_16((a1 << 1) ^ b, rc);
  a2 = red8_16((a2 << 2) ^ b, rc);
  a3 = red8_16((a3 << 3) ^ b, rc);
  a4 = red8_16((a4 << 4) ^ b, rc);
}

__device__ __forceinline__ uint32_t word_of(const uint4& v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

__global__ void __launch_bounds__(kG8Threads) sig8_kernel(const uint8_t* __restrict__ arena,
                                                          const uint64_t* __restrict__ off, uint64_t n,
                                                          uint64_t* __restrict__ sig_out) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* red = reinterpret_cast<uint32_t*>(smem);
  init_red8_tables(red, red + kRedWords);           // ends with __syncthreads()
  const RedCursor rc = red_cursor(red);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t s0 = off[i], e = off[i + 1];
    uint32_t a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    if (e > s0) {
      for (uint64_t cb = (e - 1) & ~15ull;; cb -= 16) {        // aligned chunks, last one first
        const uint4 v = *reinterpret_cast<const uint4*>(arena + cb);
        const uint32_t lo = s0 > cb ? (uint32_t)(s0 - cb) : 0u;  // key bytes [lo, hi) of the chunk
        const uint32_t hi = e - cb < 16 ? (uint32_t)(e - cb) : 16u;
        if (lo == 0 && hi == 16) {
          gf8_word(v.w, a1, a2, a3, a4, rc);
          gf8_word(v.z, a1, a2, a3, a4, rc);
          gf8_word(v.y, a1, a2, a3, a4, rc);
          gf8_word(v.x, a1, a2, a3, a4, rc);
        } else {
          for (int j = (int)hi - 1; j >= (int)lo; --j)
            gf8_byte((word_of(v, j >> 2) >> (8 * (j & 3))) & 0xFFu, a1, a2, a3, a4, rc);
        }
        if (cb <= s0) break;
      }
    }
    sig_out[i] = (uint64_t)(a1 | (a2 << 8) | (a3 << 16) | (a4 << 24));
  }
}

constexpr size_t kSmemSig8 = (size_t)kRedBytes + 512 * 4;

}  // namespace algsig
