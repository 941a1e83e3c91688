// rounds.cuh -- warp-level helpers shared by the kernels: async copies,
// the split of a relation's keys over warps in equal shares of key bytes
// (+ an optional cost per key; a 32-ary search in the offsets by one warp), the offsets a warp loads for a round of 32 keys,
// the constant-multiply tables, and the geometry of the 16-byte chunk grid
// that the comparison join's string hash (baseline.cuh) walks in tiles of
// kTile bytes (a key starting at an odd byte is read funnel-shifted by one
// byte, so that its symbols sit on 16-bit boundaries).
#pragma once
#include <cstdint>

#include "gf16.cuh"

namespace algsig {

#ifndef ALGSIG_TILE_CHUNKS
#define ALGSIG_TILE_CHUNKS 16
#endif
constexpr int kTileChunks = ALGSIG_TILE_CHUNKS;       // 16-byte chunks per tile
constexpr int kTile = 16 * kTileChunks;               // bytes of realigned key per tile
constexpr int kSpanChunks = 32 * kTileChunks + 2;     // chunks of a round's span, worst case
// one 16-byte pad per tile-length of span, so that tiles kTile bytes apart hit different banks
constexpr int kBufBytes = 16 * (kSpanChunks + (kSpanChunks + kTileChunks - 1) / kTileChunks) + 16;
constexpr uint32_t kFull = 0xFFFFFFFFu;

// g_log / g_alog: GF(2^16) logarithm / antilogarithm of x, defined (and set
// up once per device) by the translation unit that includes this header.

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------------------
// async copy of a round's span into shared memory
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// shared-memory byte offset of span offset `rel` (16-byte pad after every kTile bytes)
__device__ __forceinline__ uint32_t padded(uint32_t rel) { return rel + (rel / (uint32_t)kTile) * 16u; }

// ---------------------------------------------------------------------------
// warp range: keys [k_lo, k_hi) whose starts fall in this warp's share of the
// key bytes, each key counting c more (static partition)
// ---------------------------------------------------------------------------

// first i in [0, n] with off[i] + c i >= target (off non-decreasing; c, a
// weight per key, 0 for a plain search in the offsets); 32-ary search by one warp
__device__ __forceinline__ uint64_t warp_lower_bound(const uint64_t* __restrict__ off, uint64_t n, uint64_t target,
                                                     uint64_t c = 0) {
  const int lane = threadIdx.x & 31;
  uint64_t lo = 0, hi = n;          // answer in [lo, hi]
  while (hi - lo > 32) {
    const uint64_t step = (hi - lo + 31) / 32;
    const uint64_t idx = lo + (uint64_t)lane * step;
    const bool below = idx <= hi && off[idx] + c * idx < target;
    const int cnt = __popc(__ballot_sync(kFull, below));   // lanes 0..cnt-1 are below
    if (cnt == 0) { hi = lo; break; }
    const uint64_t nlo = lo + (uint64_t)(cnt - 1) * step;
    const uint64_t nhi = lo + (uint64_t)cnt * step;
    lo = nlo + 1;                    // off[nlo] < target
    hi = nhi < hi ? nhi : hi;
    if (lo > hi) lo = hi;
  }
  const uint64_t idx = lo + (uint64_t)lane;
  const bool below = idx < hi && off[idx] + c * idx < target;
  const int cnt = __popc(__ballot_sync(kFull, below));
  return lo + (uint64_t)cnt;
}

// The keys [k_lo, k_hi) of warp `warp` of nwarps: equal shares of the work
// bytes + c per key (c = 0: of the key bytes).
__device__ __forceinline__ void warp_key_range(const uint64_t* __restrict__ off, uint64_t n, uint64_t warp,
                                               uint64_t nwarps, uint64_t* k_lo, uint64_t* k_hi, uint64_t c = 0) {
  const uint64_t base = off[0], total = off[n] - off[0] + c * n;
  auto cut = [&](uint64_t w) -> uint64_t {
    if (w == 0) return 0;
    if (w >= nwarps) return n;
    const unsigned __int128 t = (unsigned __int128)total * w / nwarps;
    return warp_lower_bound(off, n, base + (uint64_t)t, c);
  };
  *k_lo = cut(warp);
  *k_hi = cut(warp + 1);
  if (warp + 1 >= nwarps) *k_hi = n;
}

// ---------------------------------------------------------------------------
// round plan
// ---------------------------------------------------------------------------

// Offsets a plan needs: off[kc + lane] and off[kc + lane + 1], loaded ahead of time.
struct PlanLoad {
  uint64_t o0, o1;
};

__device__ __forceinline__ PlanLoad plan_load(const uint64_t* __restrict__ off, uint64_t kc, uint64_t k_end) {
  const uint64_t kl = kc + (uint64_t)(threadIdx.x & 31);
  PlanLoad l;
  l.o0 = 0;
  l.o1 = 0;
  if (kl < k_end) {
    l.o0 = off[kl];
    l.o1 = off[kl + 1];
  }
  return l;
}

// Constant-multiply tables (512 entries each, two byte-indexed halves), set up
// once per device in g_const: c_k^(2^s) = x^(k kTile/2 2^s) for k = 1..4 and
// s = 0..3 (the cumulative-signature scans), then x^-32.
constexpr int kConstCount = 17;                       // 16 scan constants (s = 0..3) + x^-32
constexpr int kScanLevels = 4;                         // c_k^(2^s) tables kept for s < kScanLevels
constexpr int kConstEntries = kConstCount * 512;
constexpr int kConstBytes = kConstEntries * 2;

// multiply by the constant whose table starts at `tab`
__device__ __forceinline__ uint32_t mulc(const uint16_t* tab, uint32_t v) {
  return (uint32_t)tab[v & 0xFFu] ^ (uint32_t)tab[256u + (v >> 8)];
}

// x^-(k lo/2) * P, component-wise; inv32: the table of x^-32
template <class Cursor>
__device__ __forceinline__ uint64_t lo_correct_inv(const uint16_t* inv32, uint64_t P, uint32_t lo, const Cursor& rc) {
  uint64_t out = 0;
#pragma unroll
  for (int k = 1; k <= 4; k++) {
    const uint32_t m = (uint32_t)k * (lo >> 1);                 // <= 28
    const uint32_t d = mulc(inv32, (uint32_t)(P >> (16 * (k - 1))) & 0xFFFFu);
    const uint64_t E = (uint64_t)d << (32 - m);                 // d x^(32-m), < 2^48
    const uint32_t r1 = red32((uint32_t)(E >> 16), rc);
    const uint32_t r = red32(((uint32_t)E & 0xFFFFu) ^ (r1 << 16), rc);
    out |= (uint64_t)r << (16 * (k - 1));
  }
  return out;
}

}  // namespace algsig
