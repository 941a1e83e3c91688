// baseline.cuh -- the comparison join: a GPU hash join on full strings.
//
// This is the simple hash join the paper compares against (Section 2, and the
// "a.equal(b)" comparison of Section 4.3), built with the same machinery as
// the signature join so that the two differ only in the method:
//   * key hash: a 64-bit hash of all of a key's bytes, H = fmix64(len * C ^
//     XOR_i fmix64(w_i ^ (i * G + D))) over the key's 8-byte words w_i (the
//     last one zero-padded).  Each word is mixed with its index, so the words
//     can be hashed in any order: tiles of 256 key bytes are hashed by the
//     lanes of a warp from a shared-memory copy of the round's span (the tile
//     walk of rounds.cuh) and joined with a segmented XOR.
//   * table: open addressing, linear probing over the same capacity as the
//     signature table; a slot is one uint64 (hash tag << 32 | R row), all ones
//     when empty.
//   * probe: every S key walks its bucket sequence until an empty slot.  In
//     the plain variant every visited slot costs a length check and, when the
//     lengths agree, a full byte comparison; in the tagged variant (honesty
//     control) a slot is compared only when its 32-bit hash tag matches.
#pragma once
#include <cstdint>

#include "rounds.cuh"

namespace algsig {

constexpr int kBTile = 256;                         // key bytes per lane and round
constexpr int kBTileWords = kBTile / 8;
constexpr int kBSpanChunks = 32 * (kBTile / 16) + 2;
constexpr int kBBufBytes = 16 * (kBSpanChunks + (kBSpanChunks + 15) / 16) + 16;

__device__ __forceinline__ uint32_t bpadded(uint32_t rel) { return rel + (rel / (uint32_t)kBTile) * 16u; }

__device__ __forceinline__ uint64_t word_mix(uint64_t w, uint64_t i) {
  return fmix64(w ^ (i * 0x9E3779B97F4A7C15ull + 0xD6E8FEB86659FD93ull));
}

__device__ __forceinline__ uint64_t key_tiles_b(uint64_t len) { return len == 0 ? 1 : (len + kBTile - 1) / kBTile; }

struct BPlan {
  uint64_t tstart;     // arena offset of the lane's tile
  uint64_t kstart, klen;
  uint32_t tile, tlen;
  int q;
  uint32_t slot0, rq;
  bool active;
  bool valid;
  uint64_t kc, kc_next, tc_next, span_lo, span_hi;
  bool carries;
  uint32_t s31;
};

__device__ __forceinline__ BPlan bplan_round(const PlanLoad& L, uint64_t kc, uint64_t k_end, uint64_t tc) {
  BPlan p;
  p.valid = kc < k_end;
  p.kc = kc;
  const int lane = threadIdx.x & 31;
  const uint64_t kl = kc + (uint64_t)lane;
  const bool have = p.valid && kl < k_end;
  const uint64_t sl = L.o0, ll = L.o1 - L.o0;
  uint32_t rc = 0;
  if (have) {
    uint64_t nt = key_tiles_b(ll);
    if (lane == 0) nt -= tc;
    rc = nt > 33 ? 33u : (uint32_t)nt;
  }
  uint32_t cum = rc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, cum, d);
    if (lane >= d) cum += t;
  }
  const uint32_t total = __shfl_sync(kFull, cum, 31);
  int q = 0;
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const uint32_t cv = __shfl_sync(kFull, cum, q + d - 1);
    if (cv <= (uint32_t)lane) q += d;
  }
  p.active = p.valid && (uint32_t)lane < total;
  const uint32_t cq = __shfl_sync(kFull, cum, q);
  p.rq = __shfl_sync(kFull, rc, q);
  p.kstart = __shfl_sync(kFull, sl, q);
  p.klen = __shfl_sync(kFull, ll, q);
  p.q = q;
  p.slot0 = cq - p.rq;
  const uint64_t tile = (uint64_t)((uint32_t)lane - p.slot0) + (q == 0 ? tc : 0);
  p.tile = (uint32_t)tile;
  const uint64_t toff = tile * (uint64_t)kBTile;
  const uint64_t rest = p.klen > toff ? p.klen - toff : 0;
  p.tlen = p.active ? (rest < (uint64_t)kBTile ? (uint32_t)rest : (uint32_t)kBTile) : 0u;
  p.tstart = p.kstart + toff;
  const int last = (int)(total < 32u ? total : 32u) - 1;
  const uint64_t sa = __shfl_sync(kFull, p.tstart, 0);
  const uint64_t sb = __shfl_sync(kFull, p.tstart + p.tlen, last < 0 ? 0 : last);
  p.span_lo = sa & ~15ull;
  p.span_hi = (sb + 15) & ~15ull;
  if (!p.valid) {
    p.kc_next = kc; p.tc_next = tc; p.carries = false; p.s31 = 0;
  } else if (total <= 32u) {
    p.kc_next = kc + (k_end - kc < 32 ? k_end - kc : 32);
    p.tc_next = 0; p.carries = false; p.s31 = 0;
  } else {
    const int q31 = __shfl_sync(kFull, q, 31);
    const uint32_t s31 = __shfl_sync(kFull, p.slot0, 31);
    const uint32_t c31 = __shfl_sync(kFull, cq, 31);
    if (c31 == 32u) {
      p.kc_next = kc + (uint64_t)q31 + 1; p.tc_next = 0; p.carries = false; p.s31 = 0;
    } else {
      p.kc_next = kc + (uint64_t)q31;
      p.tc_next = (q31 == 0 ? tc : 0) + (uint64_t)(32u - s31);
      p.carries = true; p.s31 = s31;
    }
  }
  return p;
}

__device__ __forceinline__ void bissue_span(uint8_t* buf, const uint8_t* __restrict__ arena, const BPlan& p) {
  if (p.valid) {
    const int lane = threadIdx.x & 31;
    const uint32_t nchunks = (uint32_t)((p.span_hi - p.span_lo) >> 4);
    const uint8_t* src = arena + p.span_lo;
    for (uint32_t i = (uint32_t)lane; i < nchunks; i += 32)
      cp_async16(buf + 16 * (i + i / (uint32_t)(kBTile / 16)), src + 16 * i);
  }
  cp_async_commit();
}

// 8-byte aligned word at span offset rel (a multiple of 8) from the padded copy
__device__ __forceinline__ uint64_t bword(const uint8_t* buf, uint32_t rel) {
  return *reinterpret_cast<const uint64_t*>(buf + bpadded(rel & ~15u) + (rel & 8u));
}

// XOR of the mixed key words of the lane's tile
__device__ __forceinline__ uint64_t btile_hash(const uint8_t* buf, const BPlan& p) {
  if (p.tlen == 0) return 0;
  const uint32_t a8 = (uint32_t)(p.tstart & 7u);
  const uint32_t rel0 = (uint32_t)((p.tstart - a8) - p.span_lo);
  const uint32_t nw = (p.tlen + 7) >> 3;
  const uint64_t wi0 = (uint64_t)p.tile * kBTileWords;
  uint64_t acc = 0;
  uint64_t cur = bword(buf, rel0);             // aligned word 0 holds tile byte 0
  for (uint32_t w = 0; w < nw; ++w) {
    uint64_t v;
    if (a8) {                                  // tile bytes [8w, 8w+8) span aligned words w, w+1
      const uint64_t nxt = 8 * (w + 1) < a8 + p.tlen ? bword(buf, rel0 + 8 * (w + 1)) : 0ull;
      v = (cur >> (8 * a8)) | (nxt << (64 - 8 * a8));
      cur = nxt;
    } else {
      v = cur;
      if (w + 1 < nw) cur = bword(buf, rel0 + 8 * (w + 1));
    }
    const uint32_t left = p.tlen - 8 * w;
    if (left < 8) v &= (1ull << (8 * left)) - 1ull;
    acc ^= word_mix(v, wi0 + w);
  }
  return acc;
}

__device__ __forceinline__ uint64_t key_hash_final(uint64_t acc, uint64_t len) {
  return fmix64(acc ^ (len * 0xC2B2AE3D27D4EB4Full));
}

}  // namespace algsig
