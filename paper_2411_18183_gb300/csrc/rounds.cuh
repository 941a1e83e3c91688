// rounds.cuh -- the warp-level tile walk shared by the signature and probe
// kernels.
//
// Geometry.  A key starting at arena byte ks is read on the 16-byte chunk grid
// of the arena.  If ks is odd, the byte stream is funnel-shifted by one byte
// so that the key's symbols sit on 16-bit boundaries ("realigned" stream);
// the key then starts at the even offset lo = (ks & 15) - (ks & 1) of its
// first realigned chunk.  A tile is kTileChunks realigned chunks of that grid
// (kTile bytes): tile j of a key covers realigned chunks [j, j+1) * kTileChunks
// (the first tile starts at lo, the last ends with the key), so interior tiles
// read exactly kTileChunks aligned chunks.  An empty key has one empty tile.
//
// Rounds.  A warp owns a contiguous, byte-balanced range of keys and walks
// their tiles in rounds of 32 (one per lane).  The 32 tiles of a round are
// consecutive in the arena, so a round reads one contiguous span; cp.async
// copies it to shared memory two rounds ahead of the arithmetic.  In shared
// memory a 16-byte pad follows every kTile bytes of span, so that the lanes of
// one key, whose tiles are kTile bytes apart, read different banks.
//
// Combination.  Each lane computes its tile's signature relative to the
// tile's first slot (Horner over 16-byte chunks, gf16.cuh) and moves it to the
// tile's place in the key by a multiplication with x^(k (kTile/2 j - lo/2)) through
// log/antilog tables; the log lookups are issued before the next round is
// planned, which hides their latency.  Tiles of one key sit in consecutive
// lanes: a segmented XOR gathers them in the key's first lane of the round,
// and a key that continues into the next round carries its partial signature
// there.  Every key's signature is finished by exactly one lane.
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
// arena bytes (byte-balanced static partition)
// ---------------------------------------------------------------------------

// first i in [0, n] with off[i] >= target (off non-decreasing); 32-ary search by one warp
__device__ __forceinline__ uint64_t warp_lower_bound(const uint64_t* __restrict__ off, uint64_t n, uint64_t target) {
  const int lane = threadIdx.x & 31;
  uint64_t lo = 0, hi = n;          // answer in [lo, hi]
  while (hi - lo > 32) {
    const uint64_t step = (hi - lo + 31) / 32;
    const uint64_t idx = lo + (uint64_t)lane * step;
    const bool below = idx <= hi && off[idx] < target;
    const int cnt = __popc(__ballot_sync(kFull, below));   // lanes 0..cnt-1 are below
    if (cnt == 0) { hi = lo; break; }
    const uint64_t nlo = lo + (uint64_t)(cnt - 1) * step;
    const uint64_t nhi = lo + (uint64_t)cnt * step;
    lo = nlo + 1;                    // off[nlo] < target
    hi = nhi < hi ? nhi : hi;
    if (lo > hi) lo = hi;
  }
  const uint64_t idx = lo + (uint64_t)lane;
  const bool below = idx < hi && off[idx] < target;
  const int cnt = __popc(__ballot_sync(kFull, below));
  return lo + (uint64_t)cnt;
}

__device__ __forceinline__ void warp_key_range(const uint64_t* __restrict__ off, uint64_t n, uint64_t warp,
                                               uint64_t nwarps, uint64_t* k_lo, uint64_t* k_hi) {
  const uint64_t base = off[0], total = off[n] - off[0];
  auto cut = [&](uint64_t w) -> uint64_t {
    if (w == 0) return 0;
    if (w >= nwarps) return n;
    const unsigned __int128 t = (unsigned __int128)total * w / nwarps;
    return warp_lower_bound(off, n, base + (uint64_t)t);
  };
  *k_lo = cut(warp);
  *k_hi = cut(warp + 1);
  if (warp + 1 >= nwarps) *k_hi = n;
}

// ---------------------------------------------------------------------------
// round plan
// ---------------------------------------------------------------------------

struct Plan {
  // per lane: the tile
  uint64_t cbase;    // arena address of the tile's first aligned chunk
  uint64_t kstart;   // start / length of the tile's key
  uint64_t klen;
  uint32_t tile;     // tile index inside the key (< 2^32 tiles per key)
  uint32_t nc;       // realigned chunks in the tile (0 for an empty key)
  uint32_t lo;       // even start offset of the key in its first realigned chunk
  uint32_t odd;      // key starts at an odd byte
  uint32_t tail_e;   // valid bytes of the tile's last chunk (16 unless it ends the key)
  bool last;         // tile ends its key
  bool active;
  int q;             // key-lane index: key = kc + q
  uint32_t slot0;    // first slot of key q in this round
  uint32_t rq;       // tiles of key q in this round and after (clamped to 33)
  // warp-uniform
  bool valid;
  uint64_t kc;               // first key of the round
  uint64_t tc;               // tiles of key kc done before the round
  uint64_t kc_next, tc_next; // walk state after the round
  uint64_t span_lo, span_hi; // 16-byte aligned arena span of the round
  bool carries;              // key of slot 31 continues into the next round
  uint32_t s31;              // its first slot
};

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

__device__ __forceinline__ uint64_t key_tiles(uint64_t ks, uint64_t len) {
  if (len == 0) return 1;
  const uint64_t lo = (ks & 15u) & ~1ull;
  return (lo + len + kTile - 1) / kTile;
}

__device__ __forceinline__ Plan plan_round(const PlanLoad& L, uint64_t kc, uint64_t k_end, uint64_t tc) {
  Plan p;
  p.valid = kc < k_end;
  p.kc = kc;
  p.tc = tc;
  const int lane = threadIdx.x & 31;
  const uint64_t kl = kc + (uint64_t)lane;
  const bool have = p.valid && kl < k_end;
  const uint64_t sl = L.o0;
  const uint64_t ll = L.o1 - L.o0;
  uint32_t rc = 0;
  if (have) {
    uint64_t nt = key_tiles(sl, ll);
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
  // owner of each lane's tile: the last key whose first tile slot is at or
  // before the lane (every loaded key has at least one tile)
  const uint32_t first = cum - rc;
  const uint32_t starts = __reduce_or_sync(kFull, rc != 0u && first < 32u ? 1u << first : 0u);
  int q = __popc(starts & ((2u << lane) - 1u)) - 1;
  if (q < 0) q = 0;
  p.active = p.valid && (uint32_t)lane < total;
  const uint32_t cq = __shfl_sync(kFull, cum, q);
  p.rq = __shfl_sync(kFull, rc, q);
  p.kstart = __shfl_sync(kFull, sl, q);
  p.klen = __shfl_sync(kFull, ll, q);
  p.q = q;
  p.slot0 = cq - p.rq;
  const uint64_t tile = (uint64_t)((uint32_t)lane - p.slot0) + (q == 0 ? tc : 0);
  p.tile = (uint32_t)tile;
  // tile geometry
  const uint32_t a = (uint32_t)(p.kstart & 15u);
  p.odd = a & 1u;
  p.lo = a - p.odd;
  const uint64_t kbase = p.kstart - a;
  const uint64_t C = p.klen == 0 ? 0 : (p.lo + p.klen + 15) >> 4;       // realigned chunks of the key
  const uint64_t c0 = tile * (kTileChunks);
  const uint64_t rest = C > c0 ? C - c0 : 0;
  p.nc = p.active ? (uint32_t)(rest < (uint64_t)(kTileChunks) ? rest : (uint64_t)(kTileChunks)) : 0u;
  p.last = c0 + (kTileChunks) >= C;
  p.tail_e = p.last && p.klen ? (uint32_t)(p.lo + p.klen - 16 * (C - 1)) : 16u;
  p.cbase = kbase + 16 * c0;
  // tile's arena byte range: [max(ks, cbase + odd), min(ks + len, cbase + 128 + odd))
  const uint64_t tb = c0 == 0 ? p.kstart : p.cbase + p.odd;
  const uint64_t te_full = p.cbase + kTile + p.odd;
  const uint64_t te = p.kstart + p.klen < te_full ? p.kstart + p.klen : te_full;
  // span of the round: first active tile's first chunk .. last active tile's end
  const int last = (int)(total < 32u ? total : 32u) - 1;
  const uint64_t sa = __shfl_sync(kFull, tb, 0);
  const uint64_t sb = __shfl_sync(kFull, p.active ? te : tb, last < 0 ? 0 : last);
  p.span_lo = sa & ~15ull;
  p.span_hi = (sb + 15) & ~15ull;
  // advance the walk
  if (!p.valid) {
    p.kc_next = kc; p.tc_next = tc; p.carries = false; p.s31 = 0;
  } else if (total <= 32u) {
    const uint64_t loaded = k_end - kc < 32 ? k_end - kc : 32;
    p.kc_next = kc + loaded;
    p.tc_next = 0;
    p.carries = false;
    p.s31 = 0;
  } else {
    const int q31 = __shfl_sync(kFull, q, 31);
    const uint32_t s31 = __shfl_sync(kFull, p.slot0, 31);
    const uint32_t c31 = __shfl_sync(kFull, cq, 31);
    if (c31 == 32u) {
      p.kc_next = kc + (uint64_t)q31 + 1;
      p.tc_next = 0;
      p.carries = false;
      p.s31 = 0;
    } else {
      p.kc_next = kc + (uint64_t)q31;
      p.tc_next = (q31 == 0 ? tc : 0) + (uint64_t)(32u - s31);
      p.carries = true;
      p.s31 = s31;
    }
  }
  return p;
}

// copy the round's span into `buf` (padded layout), one commit group per call.
// Lane l copies the span's chunks l + 32 j; with kTileChunks dividing 32 their
// padded places are kCopyStride bytes apart, so the copies of a lane take
// fixed offsets from two base addresses (a fall-through switch on the count).
static_assert(32 % kTileChunks == 0, "tiles must divide a warp's 32 chunks");
constexpr uint32_t kCopyStride = 16u * (32u + 32u / kTileChunks);
static_assert(kSpanChunks <= 17 * 32, "span copies: at most 17 per lane");
__device__ __forceinline__ void issue_span(uint8_t* buf, const uint8_t* __restrict__ arena, const Plan& p) {
  if (p.valid) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nchunks = (uint32_t)((p.span_hi - p.span_lo) >> 4);
    const uint32_t cnt = nchunks > lane ? (nchunks - lane + 31u) >> 5 : 0u;
    uint8_t* d = buf + 16u * (lane + lane / (uint32_t)kTileChunks);
    const uint8_t* g = arena + p.span_lo + 16u * lane;
#define ALGSIG_COPY(j) case (j) + 1: cp_async16(d + kCopyStride * (j), g + 512u * (j));
    switch (cnt) {
      ALGSIG_COPY(16) ALGSIG_COPY(15) ALGSIG_COPY(14) ALGSIG_COPY(13) ALGSIG_COPY(12) ALGSIG_COPY(11)
      ALGSIG_COPY(10) ALGSIG_COPY(9) ALGSIG_COPY(8) ALGSIG_COPY(7) ALGSIG_COPY(6) ALGSIG_COPY(5)
      ALGSIG_COPY(4) ALGSIG_COPY(3) ALGSIG_COPY(2) ALGSIG_COPY(1) ALGSIG_COPY(0)
      default: break;
    }
#undef ALGSIG_COPY
  }
  cp_async_commit();
}

// ---------------------------------------------------------------------------
// signature of one tile from the shared-memory copy of its span
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint4 chunk_at(const uint8_t* buf, uint32_t rel) {
  return *reinterpret_cast<const uint4*>(buf + padded(rel));
}

// keep bytes [b0, 16) of a chunk given as two 64-bit halves
__device__ __forceinline__ void keep_from(uint32_t b0, uint64_t& lo64, uint64_t& hi64) {
  lo64 = b0 >= 8 ? 0ull : (~0ull << (8 * b0));
  hi64 = b0 <= 8 ? ~0ull : (~0ull << (8 * (b0 - 8)));
}
// keep bytes [0, e) of a chunk, 1 <= e <= 16
__device__ __forceinline__ void keep_below(uint32_t e, uint64_t& lo64, uint64_t& hi64) {
  lo64 = e >= 8 ? ~0ull : ((1ull << (8 * e)) - 1ull);
  hi64 = e >= 16 ? ~0ull : (e <= 8 ? 0ull : ((1ull << (8 * (e - 8))) - 1ull));
}

// Unreduced-free tile signature: a_k = sum over the tile's slots t of q_t x^(k t)
// (slot 0 = first byte pair of the tile's first realigned chunk), reduced to 16 bits.
template <int NCOMP = 4, class Cursor>
__device__ __forceinline__ void tile_accumulate(const uint8_t* buf, uint64_t span_lo, const Plan& p,
                                                const Cursor& redl, uint32_t& a1, uint32_t& a2,
                                                uint32_t& a3, uint32_t& a4) {
  a1 = a2 = a3 = a4 = 0;
  if (p.nc == 0) return;
  const uint32_t rel0 = (uint32_t)(p.cbase - span_lo);
  const uint32_t sh = p.odd * 8u;
  // head / tail masks of the first / last chunk
  uint64_t hl = ~0ull, hh = ~0ull, tl = ~0ull, th = ~0ull;
  if (p.tile == 0) keep_from(p.lo, hl, hh);
  if (p.last) keep_below(p.tail_e, tl, th);
  int c = (int)p.nc - 1;
  // the odd realignment of the tile's last chunk reads the first word of the next chunk
  uint32_t nxt0 = 0;
  if (p.odd && (!p.last || p.tail_e == 16)) nxt0 = chunk_at(buf, rel0 + 16u * (uint32_t)(c + 1)).x;
  {
    const uint4 w = chunk_at(buf, rel0 + 16u * (uint32_t)c);
    uint64_t ml = tl, mh = th;
    if (c == 0) { ml &= hl; mh &= hh; }
    const uint32_t v0 = __funnelshift_r(w.x, w.y, sh) & (uint32_t)ml;
    const uint32_t v1 = __funnelshift_r(w.y, w.z, sh) & (uint32_t)(ml >> 32);
    const uint32_t v2 = __funnelshift_r(w.z, w.w, sh) & (uint32_t)mh;
    const uint32_t v3 = __funnelshift_r(w.w, nxt0, sh) & (uint32_t)(mh >> 32);
    horner_chunk<NCOMP>(v0, v1, v2, v3, a1, a2, a3, a4, redl);
    nxt0 = w.x;
  }
  for (--c; c >= 1; --c) {
    const uint4 w = chunk_at(buf, rel0 + 16u * (uint32_t)c);
    horner_chunk<NCOMP>(__funnelshift_r(w.x, w.y, sh), __funnelshift_r(w.y, w.z, sh), __funnelshift_r(w.z, w.w, sh),
                 __funnelshift_r(w.w, nxt0, sh), a1, a2, a3, a4, redl);
    nxt0 = w.x;
  }
  if (c == 0) {
    const uint4 w = chunk_at(buf, rel0);
    const uint32_t v0 = __funnelshift_r(w.x, w.y, sh) & (uint32_t)hl;
    const uint32_t v1 = __funnelshift_r(w.y, w.z, sh) & (uint32_t)(hl >> 32);
    const uint32_t v2 = __funnelshift_r(w.z, w.w, sh) & (uint32_t)hh;
    const uint32_t v3 = __funnelshift_r(w.w, nxt0, sh) & (uint32_t)(hh >> 32);
    horner_chunk<NCOMP>(v0, v1, v2, v3, a1, a2, a3, a4, redl);
  }
}

// ---------------------------------------------------------------------------
// Combination of the tiles of a round
// ---------------------------------------------------------------------------
//
// Tile values A_j (relative to each tile's first slot) of one key are joined
// by Horner's rule with the constant c_k = x^(k kTile/2):
//     B = sum_i c_k^i A_(j0+i)
// computed as a reverse segmented scan over the lanes of the key (log2(32)
// doubling steps, step s multiplying by c_k^(2^s)).  A multiplication by a
// constant C is two lookups in a 512-entry table (low byte, high byte) held in
// shared memory: tables for c_k^(2^s) (k = 1..4, s = 0..3; s = 4 applies the
// s = 3 table twice) and for x^-32.
//
// A key whose tile 0 lies in the round gets its signature from B directly; the
// shift of its first symbol to slot lo/2 of the chunk grid is undone once per
// key by x^-(k lo/2).  A key that continues from an earlier round needs
// x^(k kTile/2 j0) B with a variable j0: that product goes through the
// log/antilog tables in global memory and is finished one round later, so the
// lookups overlap the next round's arithmetic.

constexpr int kConstCount = 17;                       // 16 scan constants (s = 0..3) + x^-32
constexpr int kScanLevels = 4;                         // c_k^(2^s) tables kept for s < kScanLevels
constexpr int kConstEntries = kConstCount * 512;
constexpr int kConstBytes = kConstEntries * 2;

// multiply by the constant whose table starts at `tab`
__device__ __forceinline__ uint32_t mulc(const uint16_t* tab, uint32_t v) {
  return (uint32_t)tab[v & 0xFFu] ^ (uint32_t)tab[256u + (v >> 8)];
}

// component-wise multiply of a packed signature by c_k^(2^s)
__device__ __forceinline__ uint64_t mul_scan(const uint16_t* ctab, uint64_t v, int s) {
  uint64_t r = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    uint32_t c = (uint32_t)(v >> (16 * k)) & 0xFFFFu;
    if (s < kScanLevels) {
      c = mulc(ctab + (size_t)(k * kScanLevels + s) * 512, c);
    } else {                                           // c_k^16 = (c_k^8)^2
      const uint16_t* t = ctab + (size_t)(k * kScanLevels + kScanLevels - 1) * 512;
      c = mulc(t, mulc(t, c));
    }
    r |= (uint64_t)c << (16 * k);
  }
  return r;
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
template <class Cursor>
__device__ __forceinline__ uint64_t lo_correct(const uint16_t* ctab, uint64_t P, uint32_t lo, const Cursor& rc) {
  return lo_correct_inv(ctab + (size_t)(4 * kScanLevels) * 512, P, lo, rc);
}

// packed tile value of a lane
__device__ __forceinline__ uint64_t pack4(uint32_t a1, uint32_t a2, uint32_t a3, uint32_t a4) {
  return (uint64_t)a1 | ((uint64_t)a2 << 16) | ((uint64_t)a3 << 32) | ((uint64_t)a4 << 48);
}

// Reverse segmented scan: the first lane of every key group ends with B.
__device__ __forceinline__ uint64_t scan_round(const Plan& p, uint64_t V, const uint16_t* ctab) {
  const int lane = threadIdx.x & 31;
  const int g = p.active ? p.q : 32 + lane;
  const uint32_t room = 32u - p.slot0;
  const uint32_t gsize = p.active ? (p.rq < room ? p.rq : room) : 1u;
  const uint32_t gmax = __reduce_max_sync(kFull, gsize);
  for (int s = 0; (1u << s) < gmax; ++s) {
    const uint64_t o = __shfl_down_sync(kFull, V, 1u << s);
    const int og = __shfl_down_sync(kFull, g, 1u << s);
    if (lane + (1 << s) < 32 && og == g) V ^= mul_scan(ctab, o, s);
  }
  return V;
}

// The deferred product x^(k e) B of a continuing key (see above), held by
// every lane (warp-uniform).
struct Pending {
  bool valid;
  bool complete;     // the key ends in the round that created this
  uint64_t key;
  uint64_t carry;    // partial signature of the key before that round
  uint32_t lo;
  uint32_t l1, l2, l3, l4;   // log(B_k) as loaded (then: antilogs of log(B_k) + k e)
  uint32_t e1;               // e mod 65535
  uint32_t zero;             // bit k-1: B_k = 0
};

__device__ __forceinline__ uint32_t alog_of(uint32_t l) {
  if (l >= kOrder) l -= kOrder;
  return __ldg(&g_alog[l]);
}

// start the product x^(k e) B: the log loads only; nothing waits for them
// before pending_alogs, one round later
__device__ __forceinline__ void pending_logs(Pending& pd, uint64_t B, uint64_t tile0) {
  pd.e1 = (uint32_t)(tile0 % kOrder) * (uint32_t)(kTile / 2) % kOrder;
  const uint32_t b1 = (uint32_t)B & 0xFFFFu, b2 = (uint32_t)(B >> 16) & 0xFFFFu;
  const uint32_t b3 = (uint32_t)(B >> 32) & 0xFFFFu, b4 = (uint32_t)(B >> 48) & 0xFFFFu;
  pd.zero = (b1 ? 0u : 1u) | (b2 ? 0u : 2u) | (b3 ? 0u : 4u) | (b4 ? 0u : 8u);
  pd.l1 = __ldg(&g_log[b1]);
  pd.l2 = __ldg(&g_log[b2]);
  pd.l3 = __ldg(&g_log[b3]);
  pd.l4 = __ldg(&g_log[b4]);
}
__device__ __forceinline__ void pending_alogs(Pending& pd) {
  const uint32_t e1 = pd.e1;
  uint32_t e2 = e1 * 2u; if (e2 >= kOrder) e2 -= kOrder;
  uint32_t e3 = e2 + e1; if (e3 >= kOrder) e3 -= kOrder;
  uint32_t e4 = e2 * 2u; if (e4 >= kOrder) e4 -= kOrder;
  pd.l1 = (pd.zero & 1u) ? 0u : alog_of(pd.l1 + e1);
  pd.l2 = (pd.zero & 2u) ? 0u : alog_of(pd.l2 + e2);
  pd.l3 = (pd.zero & 4u) ? 0u : alog_of(pd.l3 + e3);
  pd.l4 = (pd.zero & 8u) ? 0u : alog_of(pd.l4 + e4);
}
__device__ __forceinline__ uint64_t pending_value(const Pending& pd) {
  return pd.carry ^ pack4(pd.l1, pd.l2, pd.l3, pd.l4);
}

}  // namespace algsig
