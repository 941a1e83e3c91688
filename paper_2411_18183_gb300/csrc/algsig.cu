// algsig.cu -- sm_103a kernels and C ABI of the algebraic-signature equi-join.
//
// Pipeline of one join T = Join(R, S) (Figure 2 of the paper):
//   1. signatures of R      sig_key_kernel (Section 3.1; sigkey.cuh)
//   2. build H_sign on R    build_kernel   (Figure 2, formula 3)
//   3. probe with S         sig_key_kernel on S, then verify_kernel: table
//                           walk, byte-exact verification, output compaction
//                           (formulas 4-5)
// sig_key_kernel computes one key per lane (keys grouped by length, a
// bit-sliced Horner state for three of the four components).  A batch whose
// joins' rows are not one run of the relation uses sig_kernel, the warp tile
// walk of rounds.cuh over the joins' row ranges.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/algsig.h"
#include "loopbounds.h"
#include <nvtx3/nvToolsExt.h>
#include "gf16.cuh"

namespace algsig {
// GF(2^16) logarithm / antilogarithm of x, set up once per device.
__device__ uint16_t g_log[65536];
__device__ uint16_t g_alog[65536];
// constant-multiply tables of the tile combination (rounds.cuh), set up once per device
__device__ uint16_t g_const[17 * 512];
// image of the shared-memory reduction tables (gf16.cuh: 256 rows, each entry
// replicated once per bank), set up once per device and copied by the blocks
// that need the tables, so that no block computes them
__device__ uint4 g_red_img[256 * 64 / 4];
}  // namespace algsig

#include "rounds.cuh"
static_assert(algsig::kConstEntries == 17 * 512, "g_const holds the combination tables");
#include "baseline.cuh"

namespace algsig {

#ifndef ALGSIG_WARPS
#define ALGSIG_WARPS 8
#endif
constexpr int kWarpsPerBlock = ALGSIG_WARPS;
constexpr int kThreads = 32 * kWarpsPerBlock;   // one block per SM
constexpr uint64_t kEmpty = ~0ull;              // empty hash slot
constexpr uint32_t kFlagTableFull = 1u;
constexpr uint64_t kMaxPrefixLen = 0xFFFFFFF0ull;  // the prefix join's L: one prefix block of at most this many bytes
constexpr int kMaxDevices = 64;

// shared memory: reduction tables | their scratch | per-warp double buffers | per-warp pair buffers
constexpr size_t kSmemTables = (size_t)kRedBytes + 512 * 4;
constexpr size_t kSmemBufs = (size_t)kWarpsPerBlock * 2 * kBufBytes;
constexpr size_t kSmemSig = kSmemTables + kConstBytes + kSmemBufs;
static_assert(kConstEntries == 17 * 512, "constant table size");

// ----------------------------------------------------------------------------
// Batches of joins
// ----------------------------------------------------------------------------
//
// A batch runs independent joins whose relations are row ranges of one packed
// R and one packed S relation (for example a pool of resident requests).  The
// kernels work on the virtual concatenation of the batch's ranges: virtual R
// row v of join j is actual row r_begin + (v - vr); signatures are stored by
// virtual row.  A single join is the batch of one join covering all rows.
// Join j owns the table slots [slot_off, slot_off + mask] and the output
// region [pair_off, pair_off + pair_cap) with counter counts[j].  Descriptor
// nj (one past the last) holds the totals: vr = rows of R, vs = rows of S,
// vbr / vbs = key bytes of R / S.
struct BatchJoin {
  uint64_t r_begin, r_end, s_begin, s_end;   // actual rows
  uint64_t vr, vs;                           // first virtual R / S row
  uint64_t vbr, vbs;                         // first virtual R / S key byte (set on the device)
  uint64_t slot_off, mask;
  uint64_t pair_off, pair_cap;
};

// join of virtual row v: the last j with v_j <= v (joins with no rows are skipped)
template <bool S_SIDE>
__device__ __forceinline__ int join_of_virtual(const BatchJoin* __restrict__ J, int nj, uint64_t v) {
  int lo = 0, hi = nj - 1, ans = 0;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const uint64_t b = S_SIDE ? __ldg(&J[mid].vs) : __ldg(&J[mid].vr);
    if (b <= v) { ans = mid; lo = mid + 1; } else { hi = mid - 1; }
  }
  return ans;
}

// Work of a side's virtual rows up to join j's first: its key bytes + c per row
template <bool S_SIDE>
__device__ __forceinline__ uint64_t vcost_of_join(const BatchJoin* __restrict__ J, int j, uint64_t c) {
  return S_SIDE ? __ldg(&J[j].vbs) + c * __ldg(&J[j].vs) : __ldg(&J[j].vbr) + c * __ldg(&J[j].vr);
}

// join whose share of the work holds the point `t` (last j with vcost_j <= t)
template <bool S_SIDE>
__device__ __forceinline__ int join_of_vcost(const BatchJoin* __restrict__ J, int nj, uint64_t t, uint64_t c) {
  int lo = 0, hi = nj - 1, ans = 0;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    if (vcost_of_join<S_SIDE>(J, mid, c) <= t) { ans = mid; lo = mid + 1; } else { hi = mid - 1; }
  }
  return ans;
}

// virtual byte starts of every join's keys: one block, prefix over joins
__global__ void batch_bytes_kernel(BatchJoin* J, int nj, const uint64_t* __restrict__ offR,
                                   const uint64_t* __restrict__ offS) {
  __shared__ uint64_t carry_r, carry_s;
  __shared__ uint64_t wr[32], wsum[32];
  if (threadIdx.x == 0) { carry_r = 0; carry_s = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < nj; base += blockDim.x) {
    const int j = base + (int)threadIdx.x;
    uint64_t br = 0, bs = 0;
    if (j < nj) {
      br = offR ? offR[J[j].r_end] - offR[J[j].r_begin] : 0;
      bs = offS ? offS[J[j].s_end] - offS[J[j].s_begin] : 0;
    }
    uint64_t ir = br, is = bs;                     // inclusive warp scans
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t tr = __shfl_up_sync(kFull, ir, d), ts = __shfl_up_sync(kFull, is, d);
      if (lane >= d) { ir += tr; is += ts; }
    }
    if (lane == 31) { wr[w] = ir; wsum[w] = is; }
    __syncthreads();
    if (threadIdx.x == 0) {                        // exclusive scan of warp totals
      uint64_t ar = carry_r, as = carry_s;
      for (int i = 0; i < nw; i++) {
        const uint64_t tr = wr[i], ts = wsum[i];
        wr[i] = ar; wsum[i] = as;
        ar += tr; as += ts;
      }
      carry_r = ar; carry_s = as;
    }
    __syncthreads();
    if (j < nj) {
      J[j].vbr = wr[w] + ir - br;
      J[j].vbs = wsum[w] + is - bs;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    J[nj].vbr = carry_r;
    J[nj].vbs = carry_s;
  }
}

// ----------------------------------------------------------------------------
// Signature kernel
// ----------------------------------------------------------------------------

// first actual key of join j whose share of the work (key bytes + c per key)
// starts at or after the point t (t inside join j's share), as a virtual row
template <bool S_SIDE>
__device__ __forceinline__ uint64_t vcut_in_join(const BatchJoin* J, const uint64_t* off, int j, uint64_t t,
                                                 uint64_t c) {
  const uint64_t b = S_SIDE ? __ldg(&J[j].s_begin) : __ldg(&J[j].r_begin);
  const uint64_t e = S_SIDE ? __ldg(&J[j].s_end) : __ldg(&J[j].r_end);
  const uint64_t v0 = S_SIDE ? __ldg(&J[j].vs) : __ldg(&J[j].vr);
  const uint64_t k = b + warp_lower_bound(off + b, e - b, off[b] + (t - vcost_of_join<S_SIDE>(J, j, c)), c);
  return v0 + (k - b);
}

}  // namespace algsig

#include "sigkey.cuh"

namespace algsig {

// Shared-memory address of the start of dynamic shared memory (one probe per
// device decides whether the tables can be addressed at the fixed 0x400).
__device__ uint32_t g_dyn_smem_base;
__global__ void dyn_smem_base_kernel() {
  extern __shared__ __align__(16) uint8_t smem[];
  if (threadIdx.x == 0) g_dyn_smem_base = (uint32_t)__cvta_generic_to_shared(smem);
}

// ----------------------------------------------------------------------------
// Hash table H_sign: open addressing, linear probing, 16-byte slots
//   word 0: the R row's full 64-bit signature
//   word 1: (min(len, 2^32 - 2) << 32) | R row; all ones when the slot is empty
// A build thread claims word 1 with atomicCAS and then writes word 0; the
// probe runs in a later kernel, so it never sees a half-written slot.
// ----------------------------------------------------------------------------

struct Slot {
  uint64_t sig;
  uint64_t key;   // (len32 << 32) | row
};

__device__ __forceinline__ uint32_t len32(uint64_t len) {
  return len < 0xFFFFFFFEull ? (uint32_t)len : 0xFFFFFFFEu;
}

// Insert R row `row` (signature sig, key length len) into the table tab[0..msk]:
// the first empty slot from its bucket on, claimed by atomicCAS on word 1; a
// walk over the whole table that finds none sets the table-full flag.
__device__ __forceinline__ void table_insert(Slot* tab, uint64_t msk, uint64_t sig, uint64_t len, uint64_t row,
                                             uint32_t* flags) {
  const uint64_t word = ((uint64_t)len32(len) << 32) | row;
  uint64_t b = sig_hash(sig, len) & msk;
  for (uint64_t step = 0; step <= msk; ++step) {
    const uint64_t cur = *(volatile const uint64_t*)(&tab[b].key);
    if (cur == kEmpty) {
      const unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(&tab[b].key),
                                                (unsigned long long)kEmpty, (unsigned long long)word);
      if (prev == kEmpty) {
        tab[b].sig = sig;
        return;
      }
    }
    b = (b + 1) & msk;
  }
  atomicOr(flags, kFlagTableFull);
}

// Insert R rows (batch: the m virtual rows of the joins).  Single join:
// J == nullptr, the table is slots[0..mask].
__global__ void build_kernel(Slot* __restrict__ slots, uint64_t mask, const uint64_t* __restrict__ sigR,
                             const uint64_t* __restrict__ offR, uint64_t m, uint32_t* __restrict__ flags,
                             const BatchJoin* __restrict__ J, int nj, uint64_t cap_len = ~0ull) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < m; v += stride) {
    Slot* tab = slots;
    uint64_t msk = mask;
    uint64_t row = v;                                 // batch: virtual row v -> actual row
    if (J) {
      const int j = join_of_virtual<false>(J, nj, v);
      row = __ldg(&J[j].r_begin) + (v - __ldg(&J[j].vr));
      tab = slots + __ldg(&J[j].slot_off);
      msk = __ldg(&J[j].mask);
    }
    const uint64_t full = offR[row + 1] - offR[row];
    const uint64_t len = full < cap_len ? full : cap_len;   // the prefix join reads keys' first cap_len bytes
    table_insert(tab, msk, sigR[v], len, row, flags);
  }
}

// The build fused into the signature kernel over R (as_join_build without
// given signatures): after each group of 32 keys has its signatures, every
// lane inserts its key.  The probe runs in a later kernel, so it never sees a
// slot whose signature word is not yet written.
struct BuildPost {
  static constexpr size_t kScratch = 0;
  Slot* slots;
  uint64_t mask;
  const uint64_t* offR;
  uint32_t* flags;
  __device__ __forceinline__ void init(uint8_t*, const uint4*) {}
  __device__ __forceinline__ void group(uint64_t kq, uint64_t sig, bool valid) {
    if (valid) table_insert(slots, mask, sig, __ldg(offR + kq + 1) - __ldg(offR + kq), kq, flags);
  }
  __device__ __forceinline__ void finish() {}
};

// ----------------------------------------------------------------------------
// Probe: table walk + byte-exact verification + output compaction.  The S
// signatures come from sig_kernel; this kernel needs no large shared memory,
// so it runs at full occupancy and hides the latency of its random accesses
// (slots, R offsets, key bytes) behind many warps.
// ----------------------------------------------------------------------------

constexpr int kVThreads = 256;
constexpr int kVWarps = kVThreads / 32;
constexpr int kVStage = 64;     // verified pairs staged per warp before one atomic append

struct VerifyParams {
  const Slot* slots;
  uint64_t mask;
  const uint8_t* arenaR;
  const uint64_t* offR;
  const uint32_t* idR;
  const uint8_t* arenaS;
  const uint64_t* offS;
  const uint32_t* idS;
  const uint64_t* sigS;
  uint64_t n;
  uint32_t* pairs;
  uint64_t cap;
  unsigned long long* count;
  int mode;                    // AS_JOIN_* (single joins)
  uint32_t* matched;           // R-side modes: bit per R row, set for every verified pair
  // batch mode (J != nullptr): per-join tables, output regions and counters
  const BatchJoin* J;
  int nj;
  unsigned long long* counts;
  uint64_t cap_len = ~0ull;    // keys compared on their first cap_len bytes (the prefix join)
};

__device__ __forceinline__ uint4 ld16(const uint8_t* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }
__device__ __forceinline__ uint64_t lo64(uint4 v) { return (uint64_t)v.x | ((uint64_t)v.y << 32); }
__device__ __forceinline__ uint64_t hi64(uint4 v) { return (uint64_t)v.z | ((uint64_t)v.w << 32); }
// bytes sh/8 .. sh/8 + 7 of the 16-byte pair (lo, hi), sh in {0, 8, ..., 56}
__device__ __forceinline__ uint64_t fsh64(uint64_t lo, uint64_t hi, uint32_t sh) {
  return sh ? (lo >> sh) | (hi << (64u - sh)) : lo;
}
// keep bytes [b0, b1) of an 8-byte word (0 <= b0, b1 <= 8)
__device__ __forceinline__ uint64_t bytes_mask(int b0, int b1) {
  if (b1 <= b0) return 0ull;
  const uint64_t hi = b1 >= 8 ? ~0ull : ((1ull << (8 * b1)) - 1ull);
  return hi & (~0ull << (8 * b0));
}
// Byte equality of the len-byte keys at aR + r0 and aS + s0 by the whole
// warp, 512 bytes per step, in 64-bit offsets (keys of 2^32 - 64 bytes and
// more): lane l compares the 16-byte aligned S chunk l of the step with the 16
// R bytes under it (from the two aligned R chunks that hold them).  Only
// aligned chunks that hold a key byte are read; the first R chunk is clamped
// to the arena's start (its bytes before the key are masked).
__device__ __noinline__ bool warp_equal_wide(const uint8_t* __restrict__ aR, uint64_t r0,
                                             const uint8_t* __restrict__ aS, uint64_t s0, uint64_t len) {
  const int lane = threadIdx.x & 31;
  const uint64_t se = s0 + len, re = r0 + len;
  const uint32_t d = (uint32_t)((r0 - s0) & 15u);
  const uint32_t hsel = d >> 3, sh = 8u * (d & 7u);
  for (uint64_t base = s0 & ~15ull; base < se; base += 512) {
    const uint64_t c = base + 16 * (uint64_t)lane;
    const int64_t q = (int64_t)(c + r0 - s0) - (int64_t)d;
    const uint4 sw = c < se ? ld16(aS + c) : make_uint4(0, 0, 0, 0);
    const uint4 ra = (q + 16 > (int64_t)r0 && q < (int64_t)re) ? ld16(aR + (q < 0 ? 0 : q)) : make_uint4(0, 0, 0, 0);
    const uint4 rb = (q + 16 < (int64_t)re) ? ld16(aR + q + 16) : make_uint4(0, 0, 0, 0);
    const uint64_t A0 = lo64(ra), A1 = hi64(ra), B0 = lo64(rb), B1 = hi64(rb);
    const uint64_t p0 = hsel ? A1 : A0, p1 = hsel ? B0 : A1, p2 = hsel ? B1 : B0;
    uint64_t x0 = fsh64(p0, p1, sh) ^ lo64(sw);
    uint64_t x1 = fsh64(p1, p2, sh) ^ hi64(sw);
    if (c < s0 || c + 16 > se) {
      const int b0 = c < s0 ? (int)(s0 - c) : 0;
      const int b1 = c >= se ? 0 : (c + 16 > se ? (int)(se - c) : 16);
      x0 &= bytes_mask(b0, b1 < 8 ? b1 : 8);
      x1 &= bytes_mask(b0 > 8 ? b0 - 8 : 0, b1 > 8 ? b1 - 8 : 0);
    }
    if (!__all_sync(kFull, (x0 | x1) == 0)) return false;
  }
  return true;
}

// Keys below kNarrowLen (loopbounds.h) are compared with 32-bit offsets (warp_equal).

// emask[e]: the first e bytes of a 16-byte chunk (e = 0..16), in shared memory.
__device__ __forceinline__ void fill_emask(uint4* emask) {
  for (int e = threadIdx.x; e <= 16; e += blockDim.x) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int b = e - 4 * j;
      w[j] = b <= 0 ? 0u : (b >= 4 ? ~0u : ((1u << (8 * b)) - 1u));
    }
    emask[e] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Byte equality of the len-byte keys at pR and pS (len < kNarrowLen) by the
// whole warp, 512 bytes per step.  Offsets count from the aligned chunk bS
// that holds the S key's first byte: S key bytes are [sa, sa + len); bR is
// the aligned R chunk that holds the R byte matching bS + 0 minus its
// misalignment d, so that lane l's S chunk [off, off + 16) meets the R bytes
// [off + d, off + d + 16) of the two aligned R chunks at bR + off and
// bR + off + 16, realigned by a funnel shift of d bytes (the word part of d is
// warp-uniform).  Only aligned chunks that hold a key byte are read.  Only the
// steps that hold the key's first or last byte apply byte masks.
// realigned R words of one lane for the misalignment d (word part warp-uniform)
__device__ __forceinline__ void realign_r(const uint4& ra, const uint4& rb, uint32_t d, uint32_t sh, uint32_t& r0,
                                          uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  switch (d >> 2) {                                // warp-uniform
    case 0:
      r0 = __funnelshift_r(ra.x, ra.y, sh); r1 = __funnelshift_r(ra.y, ra.z, sh);
      r2 = __funnelshift_r(ra.z, ra.w, sh); r3 = __funnelshift_r(ra.w, rb.x, sh);
      break;
    case 1:
      r0 = __funnelshift_r(ra.y, ra.z, sh); r1 = __funnelshift_r(ra.z, ra.w, sh);
      r2 = __funnelshift_r(ra.w, rb.x, sh); r3 = __funnelshift_r(rb.x, rb.y, sh);
      break;
    case 2:
      r0 = __funnelshift_r(ra.z, ra.w, sh); r1 = __funnelshift_r(ra.w, rb.x, sh);
      r2 = __funnelshift_r(rb.x, rb.y, sh); r3 = __funnelshift_r(rb.y, rb.z, sh);
      break;
    default:
      r0 = __funnelshift_r(ra.w, rb.x, sh); r1 = __funnelshift_r(rb.x, rb.y, sh);
      r2 = __funnelshift_r(rb.y, rb.z, sh); r3 = __funnelshift_r(rb.z, rb.w, sh);
      break;
  }
}

// Byte equality of the len-byte keys at pR and pS (len < kNarrowLen) by the
// whole warp, 1024 bytes per round trip: lane l compares, for each of the two
// 512-byte halves of a step, the S chunk [off, off + 16) with the R bytes
// [off + d, off + d + 16) from the two aligned R chunks at bR + off and
// bR + off + 16 (offsets from the aligned chunk bS that holds the S key's first
// byte; bR is the aligned R chunk that holds the matching R byte, minus the
// misalignment d).  Both halves' loads are issued before either is compared,
// so a key of up to 1 KB costs one memory round trip.  Only aligned chunks
// that hold a key byte are read; only the steps that hold the key's first or
// last byte apply byte masks.
// (emask[kMS * e] holds the mask of e bytes: kMS = 2 reads the first halves of
// the signature kernel's 32-byte block masks)
template <int kMS = 1>
__device__ __forceinline__ bool warp_equal(const uint8_t* __restrict__ pR, const uint8_t* __restrict__ pS,
                                           uint32_t len, const uint4* __restrict__ emask) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t sa = (uint32_t)reinterpret_cast<uintptr_t>(pS) & 15u;
  const uint32_t d = (uint32_t)(reinterpret_cast<uintptr_t>(pR) - sa) & 15u;
  const uint8_t* bS = pS - sa;
  const uint8_t* bR = pR - sa - d;
  const uint32_t sh = 8u * (d & 3u);
  const uint32_t kend = sa + len;                  // S key bytes: [sa, kend) from bS
  const uint32_t rlo = sa + d, rend = kend + d;    // R key bytes: [rlo, rend) from bR
  const uint32_t nsteps = narrow_steps(sa, len);   // offsets stay below 2^32 (len < kNarrowLen)
  for (uint32_t step = 0; step < nsteps; ++step) {
    const uint32_t base = step << 10;
    uint4 sv[2], ra[2], rb[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const uint32_t off = base + 512u * h + 16u * lane;
      sv[h] = make_uint4(0, 0, 0, 0); ra[h] = sv[h]; rb[h] = sv[h];
      if (off < kend) sv[h] = ld16(bS + off);
      if (off + 16u > rlo && off < rend) ra[h] = ld16(bR + off);
      if (off + 16u < rend) rb[h] = ld16(bR + off + 16u);
    }
    uint32_t diff = 0;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const uint32_t hb = base + 512u * h, off = hb + 16u * lane;
      uint32_t r0, r1, r2, r3;
      realign_r(ra[h], rb[h], d, sh, r0, r1, r2, r3);
      uint32_t x0 = r0 ^ sv[h].x, x1 = r1 ^ sv[h].y, x2 = r2 ^ sv[h].z, x3 = r3 ^ sv[h].w;
      if ((hb == 0u && sa != 0u) || hb + 512u > kend) {   // warp-uniform: the key's first or last byte
        const uint32_t lo = off < sa ? sa - off : 0u;
        const uint32_t hi = off < kend ? (kend - off < 16u ? kend - off : 16u) : 0u;
        const uint4 mh = emask[kMS * hi], ml = emask[kMS * lo];
        x0 &= mh.x & ~ml.x; x1 &= mh.y & ~ml.y; x2 &= mh.z & ~ml.z; x3 &= mh.w & ~ml.w;
      }
      diff |= x0 | x1 | x2 | x3;
    }
    if (__any_sync(kFull, diff != 0u)) return false;
  }
  return true;
}

// Verified pairs staged per warp as rows; their ids are looked up when the
// stage is flushed, by all lanes at once (a per-pair lookup would make the
// warp wait on memory once more per pair).
struct Stage {
  uint32_t r[kVStage];     // R row, or AS_NO_ROW
  uint64_t s[kVStage];     // S row
};

// ids of a staged pair; without ids the rows count from rb / sb
__device__ __forceinline__ uint64_t pair_ids(uint32_t r, uint64_t s, const uint32_t* idR, const uint32_t* idS,
                                             uint64_t rb, uint64_t sb) {
  const uint32_t rid = r == AS_NO_ROW ? AS_NO_ROW : (idR ? __ldg(idR + r) : (uint32_t)(r - rb));
  const uint32_t sid = idS ? __ldg(idS + s) : (uint32_t)(s - sb);
  return (uint64_t)rid | ((uint64_t)sid << 32);
}

__device__ __forceinline__ void flush_stage(const Stage& st, uint32_t np, const VerifyParams& P) {
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(P.count, (unsigned long long)np);
  base = __shfl_sync(kFull, base, 0);
  for (uint32_t i = (uint32_t)lane; i < np; i += 32) {
    const unsigned long long idx = base + i;
    if (idx < P.cap) reinterpret_cast<uint64_t*>(P.pairs)[idx] = pair_ids(st.r[i], st.s[i], P.idR, P.idS, 0, 0);
  }
  __syncwarp();
}

// flush for join j of a batch: its counter, region and capacity
__device__ __forceinline__ void flush_stage_join(const Stage& st, uint32_t np, const VerifyParams& P, int j) {
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(P.counts + j, (unsigned long long)np);
  base = __shfl_sync(kFull, base, 0);
  const uint64_t off = __ldg(&P.J[j].pair_off), cap = __ldg(&P.J[j].pair_cap);
  const uint64_t rb = __ldg(&P.J[j].r_begin), sb = __ldg(&P.J[j].s_begin);
  for (uint32_t i = (uint32_t)lane; i < np; i += 32) {
    const unsigned long long idx = base + i;
    if (idx < cap) reinterpret_cast<uint64_t*>(P.pairs)[off + idx] = pair_ids(st.r[i], st.s[i], P.idR, P.idS, rb, sb);
  }
  __syncwarp();
}

// BATCH: the S rows of a batch's joins; INNER: the plain inner join of one
// table (no output mode to test per pair)
template <bool BATCH, bool INNER = false>
__global__ void __launch_bounds__(kVThreads, 4) verify_kernel(VerifyParams P) {
  __shared__ Stage stage_all[kVWarps];
  __shared__ uint4 emask[17];
  fill_emask(emask);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  Stage& stage = stage_all[threadIdx.x >> 5];
  uint32_t np = 0;                                   // staged pairs (warp-uniform)
  int sj = -1;                                       // batch: join of the staged pairs
  constexpr bool batch = BATCH;
  const int mode = INNER ? (int)AS_JOIN_INNER : P.mode;
  const uint64_t ngroups = (P.n + 31) / 32;
  const uint64_t nwarps = (uint64_t)gridDim.x * kVWarps;
  for (uint64_t grp = (uint64_t)blockIdx.x * kVWarps + (threadIdx.x >> 5); grp < ngroups; grp += nwarps) {
    const uint64_t vi = grp * 32 + (uint64_t)lane;   // virtual S row (= actual row for one join)
    bool live = vi < P.n;
    const Slot* slots = P.slots;
    uint64_t mask = P.mask;
    uint64_t i = vi;
    int jn = 0;                                      // batch: join of the lane's S row
    if (batch && live) {
      jn = join_of_virtual<true>(P.J, P.nj, vi);
      i = __ldg(&P.J[jn].s_begin) + (vi - __ldg(&P.J[jn].vs));
      slots = P.slots + __ldg(&P.J[jn].slot_off);
      mask = __ldg(&P.J[jn].mask);
    }
    uint64_t sig = 0, start = 0, len = 0, b = 0, steps = 0;
    uint32_t l32 = 0;
    bool matched = false;                            // the lane's S row has a verified match
    const bool row_live = live;
    if (live) {
      sig = __ldg(P.sigS + vi);
      start = __ldg(P.offS + i);
      len = __ldg(P.offS + i + 1) - start;
      if (len > P.cap_len) len = P.cap_len;
      b = sig_hash(sig, len) & mask;
      l32 = len32(len);
    }
    while (__any_sync(kFull, live)) {
      bool cand = false;
      uint32_t row = 0;
      if (live) {
        const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(slots + b));
        if (v.y == kEmpty) {
          live = false;
        } else {
          if (v.x == sig && (uint32_t)(v.y >> 32) == l32) {
            cand = true;
            row = (uint32_t)v.y;
          }
          b = (b + 1) & mask;
          if (++steps > mask) live = false;
          // a slot at an even index shares its 32-byte sector with the next one: look at that one
          // too in this step (an L1 hit), unless this one was already a candidate
          if (!cand && live && (b & 1u)) {
            const ulonglong2 v2 = __ldg(reinterpret_cast<const ulonglong2*>(slots + b));
            if (v2.y == kEmpty) {
              live = false;
            } else {
              if (v2.x == sig && (uint32_t)(v2.y >> 32) == l32) {
                cand = true;
                row = (uint32_t)v2.y;
              }
              b = (b + 1) & mask;
              if (++steps > mask) live = false;
            }
          }
        }
      }
      uint32_t cm = __ballot_sync(kFull, cand);
      while (cm) {                                   // verify candidates one by one, whole warp
        const int j = __ffs(cm) - 1;
        cm &= cm - 1;
        const uint32_t rj = __shfl_sync(kFull, row, j);
        const uint32_t lj = __shfl_sync(kFull, l32, j);   // the slot holds the same length
        const uint64_t stj = __shfl_sync(kFull, start, j);
        if (cm) {                                    // the next candidate's S bytes and R offset, ahead
          const int j2 = __ffs(cm) - 1;
          const uint64_t st2 = __shfl_sync(kFull, start, j2);
          const uint32_t l2 = __shfl_sync(kFull, l32, j2);
          const uint32_t r2 = __shfl_sync(kFull, row, j2);
          const uint64_t o = 32u * (uint64_t)lane;   // one 32-byte sector per lane, the first 1 KB
          if (o < (uint64_t)l2)                     // addresses inside the key only
            asm volatile("prefetch.global.L1 [%0];" ::"l"(P.arenaS + st2 + o));
          if (lane == 0) asm volatile("prefetch.global.L1 [%0];" ::"l"(P.offR + r2));
        }
        const uint64_t rs = __ldg(P.offR + rj);
        const bool verify = batch || mode != AS_JOIN_SIG_ONLY;   // signature-only: no byte comparison
        bool eq;
        if (lj < kNarrowLen) {
          eq = !verify || warp_equal(P.arenaR + rs, P.arenaS + stj, lj, emask);
        } else {                                      // lengths that the slot's 32-bit field saturates
          const uint64_t ls = __shfl_sync(kFull, len, j);
          uint64_t lr = __ldg(P.offR + rj + 1) - rs;
          if (lr > P.cap_len) lr = P.cap_len;
          eq = lr == ls && (!verify || warp_equal_wide(P.arenaR, rs, P.arenaS, stj, ls));
        }
        if (eq) {
          const uint64_t srow = __shfl_sync(kFull, i, j);
          if (lane == j) matched = true;
          if (!batch && mode >= AS_JOIN_OUTER_R) {  // R-side modes: mark the R row
            if (lane == 0) atomicOr(P.matched + (rj >> 5), 1u << (rj & 31u));
            if (mode != AS_JOIN_OUTER_R) continue;   // rows, not pairs
          }
          if (!batch && (mode == AS_JOIN_SEMI || mode == AS_JOIN_ANTI)) continue;   // rows, not pairs
          const int jj = __shfl_sync(kFull, jn, j);
          if (batch && np && jj != sj) {              // the stage holds one join's pairs
            flush_stage_join(stage, np, P, sj);
            np = 0;
          }
          sj = jj;
          if (lane == 0) {
            stage.r[np] = rj;
            stage.s[np] = srow;
          }
          __syncwarp();
          if (++np == (uint32_t)kVStage) {
            if (batch) flush_stage_join(stage, np, P, sj); else flush_stage(stage, np, P);
            np = 0;
          }
        }
      }
    }
    if (!batch && (mode == AS_JOIN_SEMI || mode == AS_JOIN_ANTI || mode == AS_JOIN_OUTER_S)) {
      // one (AS_NO_ROW, s_id) per selected S row
      const bool emit = row_live && (mode == AS_JOIN_SEMI ? matched : !matched);
      const uint32_t em = __ballot_sync(kFull, emit);
      if (em) {
        if (np + (uint32_t)__popc(em) > (uint32_t)kVStage) {
          flush_stage(stage, np, P);
          np = 0;
        }
        if (emit) {
          const uint32_t pos = np + __popc(em & lanemask_lt());
          stage.r[pos] = AS_NO_ROW;
          stage.s[pos] = i;
        }
        np += (uint32_t)__popc(em);
        __syncwarp();
      }
    }
  }
  if (np) {
    if (batch) flush_stage_join(stage, np, P, sj); else flush_stage(stage, np, P);
  }
}

// The probe of the whole join fused into the signature kernel over S (plain
// inner join of one table): after a group of 32 keys has its signatures, the
// warp walks the table for each key and verifies the candidates as
// verify_kernel does, while the key bytes it has just streamed may still sit
// in L2.  Pairs are staged per warp in the kernel's shared scratch.
struct ProbePost {
  static constexpr size_t kScratch = sizeof(Stage);
  VerifyParams P;
  Stage* st;
  const uint4* mt;                                   // 32-byte block masks: row e keeps bytes [0, e)
  uint32_t np;
  __device__ __forceinline__ void init(uint8_t* scratch, const uint4* masks) {
    st = reinterpret_cast<Stage*>(scratch);
    mt = masks;
    np = 0;
  }
  __device__ __forceinline__ void group(uint64_t kq, uint64_t sig, bool valid) {
    const int lane = threadIdx.x & 31;
    bool live = valid;
    uint64_t start = 0, len = 0, b = 0, steps = 0;
    uint32_t l32 = 0;
    if (live) {
      start = __ldg(P.offS + kq);
      len = __ldg(P.offS + kq + 1) - start;
      b = sig_hash(sig, len) & P.mask;
      l32 = len32(len);
    }
    while (__any_sync(kFull, live)) {
      bool cand = false;
      uint32_t row = 0;
      if (live) {
        const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(P.slots + b));
        if (v.y == kEmpty) {
          live = false;
        } else {
          if (v.x == sig && (uint32_t)(v.y >> 32) == l32) {
            cand = true;
            row = (uint32_t)v.y;
          }
          b = (b + 1) & P.mask;
          if (++steps > P.mask) live = false;
          if (!cand && live && (b & 1u)) {         // the other slot of the 32-byte sector
            const ulonglong2 v2 = __ldg(reinterpret_cast<const ulonglong2*>(P.slots + b));
            if (v2.y == kEmpty) {
              live = false;
            } else {
              if (v2.x == sig && (uint32_t)(v2.y >> 32) == l32) {
                cand = true;
                row = (uint32_t)v2.y;
              }
              b = (b + 1) & P.mask;
              if (++steps > P.mask) live = false;
            }
          }
        }
      }
      uint32_t cm = __ballot_sync(kFull, cand);
      while (cm) {                                   // candidates one by one, whole warp
        const int j = __ffs(cm) - 1;
        cm &= cm - 1;
        const uint32_t rj = __shfl_sync(kFull, row, j);
        const uint32_t lj = __shfl_sync(kFull, l32, j);
        const uint64_t stj = __shfl_sync(kFull, start, j);
        if (cm) {                                    // the next candidate's S bytes and R offset, ahead
          const int j2 = __ffs(cm) - 1;
          const uint64_t st2 = __shfl_sync(kFull, start, j2);
          const uint32_t l2 = __shfl_sync(kFull, l32, j2);
          const uint32_t r2 = __shfl_sync(kFull, row, j2);
          const uint64_t o = 32u * (uint64_t)lane;
          if (o < (uint64_t)l2) asm volatile("prefetch.global.L1 [%0];" ::"l"(P.arenaS + st2 + o));
          if (lane == 0) asm volatile("prefetch.global.L1 [%0];" ::"l"(P.offR + r2));
        }
        const uint64_t rs = __ldg(P.offR + rj);
        bool eq;
        if (lj < kNarrowLen) {
          eq = warp_equal<2>(P.arenaR + rs, P.arenaS + stj, lj, mt);
        } else {
          const uint64_t ls = __shfl_sync(kFull, len, j);
          const uint64_t lr = __ldg(P.offR + rj + 1) - rs;
          eq = lr == ls && warp_equal_wide(P.arenaR, rs, P.arenaS, stj, ls);
        }
        if (eq) {
          const uint64_t srow = __shfl_sync(kFull, kq, j);
          if (lane == 0) {
            st->r[np] = rj;
            st->s[np] = srow;
          }
          __syncwarp();
          if (++np == (uint32_t)kVStage) {
            flush_stage(*st, np, P);
            np = 0;
          }
        }
      }
    }
  }
  __device__ __forceinline__ void finish() {
    if (np) flush_stage(*st, np, P);
  }
};

// The R-side output modes' rows: one (r_id, AS_NO_ROW) per R row whose bit in
// `matched` is `want` (1: semi-join rows, 0: anti-join / outer-join rows),
// appended to the pairs after those of the probe.  One warp per 32 rows: a
// ballot, one atomic per warp, lanes write their records in order.
__global__ void r_rows_kernel(const uint32_t* __restrict__ matched, uint64_t m, uint32_t want,
                              const uint32_t* __restrict__ idR, uint32_t* pairs, uint64_t cap,
                              unsigned long long* count) {
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t w = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w * 32 < m; w += nwarps) {
    const uint64_t r = w * 32 + (uint64_t)lane;
    const bool emit = r < m && ((__ldg(matched + w) >> lane) & 1u) == want;
    const uint32_t em = __ballot_sync(kFull, emit);
    if (!em) continue;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(em));
    base = __shfl_sync(kFull, base, 0);
    if (emit) {
      const unsigned long long idx = base + (unsigned long long)__popc(em & lanemask_lt());
      if (idx < cap) {
        const uint32_t rid = idR ? __ldg(idR + r) : (uint32_t)r;
        reinterpret_cast<uint64_t*>(pairs)[idx] = (uint64_t)rid | ((uint64_t)AS_NO_ROW << 32);
      }
    }
  }
}

}  // namespace algsig

#include "prefix.cuh"
#include "gf8.cuh"
#include "partition.cuh"

namespace algsig {

// ----------------------------------------------------------------------------
// Comparison join on full strings (baseline.cuh): hash, build, probe
// ----------------------------------------------------------------------------

constexpr size_t kSmemBHash = (size_t)kWarpsPerBlock * 2 * kBBufBytes;

__global__ void __launch_bounds__(kThreads, 1) bl_hash_kernel(const uint8_t* __restrict__ arena,
                                                              const uint64_t* __restrict__ off, uint64_t n,
                                                              uint64_t* __restrict__ hash_out) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint8_t* bufs = smem + (size_t)wib * 2 * kBBufBytes;
  const uint64_t warp = (uint64_t)blockIdx.x * kWarpsPerBlock + wib;
  const uint64_t nwarps = (uint64_t)gridDim.x * kWarpsPerBlock;
  uint64_t k_lo, k_hi;
  warp_key_range(off, n, warp, nwarps, &k_lo, &k_hi);
  BPlan cur = bplan_round(plan_load(off, k_lo, k_hi), k_lo, k_hi, 0);
  bissue_span(bufs, arena, cur);
  BPlan nxt = bplan_round(plan_load(off, cur.kc_next, k_hi), cur.kc_next, k_hi, cur.tc_next);
  bissue_span(bufs + kBBufBytes, arena, nxt);
  uint64_t carry = 0;
  for (int r = 0; cur.valid; ++r) {
    const PlanLoad ahead = plan_load(off, nxt.kc_next, k_hi);
    cp_async_wait_prev();
    __syncwarp();
    uint8_t* buf = bufs + (r & 1) * kBBufBytes;
    uint64_t v = cur.active ? btile_hash(buf, cur) : 0ull;
    __syncwarp();
    const BPlan nn = bplan_round(ahead, nxt.kc_next, k_hi, nxt.tc_next);
    bissue_span(buf, arena, nn);
    const int g = cur.active ? cur.q : 32 + lane;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t o = __shfl_down_sync(kFull, v, d);
      const int og = __shfl_down_sync(kFull, g, d);
      if (lane + d < 32 && og == g) v ^= o;
    }
    const bool head = cur.active && (uint32_t)lane == cur.slot0;
    if (head && cur.q == 0) v ^= carry;
    if (head && cur.slot0 + cur.rq <= 32u) hash_out[cur.kc + (uint64_t)cur.q] = key_hash_final(v, cur.klen);
    const uint64_t part = __shfl_sync(kFull, v, (int)cur.s31);
    carry = cur.carries ? part : 0ull;
    cur = nxt;
    nxt = nn;
  }
  cp_async_wait_all();
}

__global__ void bl_build_kernel(uint64_t* __restrict__ slots, uint64_t mask, const uint64_t* __restrict__ hashR,
                                uint64_t m, int tagged, uint32_t* __restrict__ flags) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; row < m; row += stride) {
    const uint64_t h = hashR[row];
    const uint64_t word = (tagged ? (h & 0xFFFFFFFF00000000ull) : 0ull) | row;
    uint64_t b = h & mask;
    bool placed = false;
    for (uint64_t step = 0; step <= mask; ++step) {
      const uint64_t cur = *(volatile const uint64_t*)(slots + b);
      if (cur == kEmpty) {
        const unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(slots + b),
                                                  (unsigned long long)kEmpty, (unsigned long long)word);
        if (prev == kEmpty) { placed = true; break; }
      }
      b = (b + 1) & mask;
    }
    if (!placed) atomicOr(flags, kFlagTableFull);
  }
}

struct BVerifyParams {
  const uint64_t* slots;
  uint64_t mask;
  int tagged;
  const uint8_t* arenaR;
  const uint64_t* offR;
  const uint32_t* idR;
  const uint8_t* arenaS;
  const uint64_t* offS;
  const uint32_t* idS;
  const uint64_t* hashS;
  uint64_t n;
  uint32_t* pairs;
  uint64_t cap;
  unsigned long long* count;
};

__global__ void __launch_bounds__(kVThreads, 4) bl_verify_kernel(BVerifyParams P) {
  __shared__ Stage stage_all[kVWarps];
  __shared__ uint4 emask[17];
  fill_emask(emask);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  Stage& stage = stage_all[threadIdx.x >> 5];
  VerifyParams VP;                                  // for flush_stage
  VP.pairs = P.pairs;
  VP.cap = P.cap;
  VP.count = P.count;
  VP.idR = P.idR;
  VP.idS = P.idS;
  uint32_t np = 0;
  const uint64_t ngroups = (P.n + 31) / 32;
  const uint64_t nwarps = (uint64_t)gridDim.x * kVWarps;
  for (uint64_t grp = (uint64_t)blockIdx.x * kVWarps + (threadIdx.x >> 5); grp < ngroups; grp += nwarps) {
    const uint64_t i = grp * 32 + (uint64_t)lane;
    bool live = i < P.n;
    uint64_t h = 0, start = 0, len = 0, b = 0, steps = 0;
    if (live) {
      h = __ldg(P.hashS + i);
      start = __ldg(P.offS + i);
      len = __ldg(P.offS + i + 1) - start;
      b = h & P.mask;
    }
    while (__any_sync(kFull, live)) {
      bool cand = false;
      uint32_t row = 0;
      uint64_t rs = 0;
      // a tag miss (tagged slots) moves on to the next slot of the same 32-byte sector in the same step,
      // as the signature join's probe does with its 16-byte slots
      while (live) {
        const uint64_t v = __ldg(P.slots + b);
        if (v == kEmpty) {
          live = false;
          break;
        }
        row = (uint32_t)v;
        const bool tag_ok = !P.tagged || (uint32_t)(v >> 32) == (uint32_t)(h >> 32);
        if (tag_ok) {
          rs = __ldg(P.offR + row);                   // every visited slot: length check
          cand = __ldg(P.offR + row + 1) - rs == len;
        }
        b = (b + 1) & P.mask;
        if (++steps > P.mask) live = false;
        if (tag_ok || (b & 3u) == 0) break;
      }
      uint32_t cm = __ballot_sync(kFull, cand);
      while (cm) {                                   // full byte comparison, whole warp
        const int j = __ffs(cm) - 1;
        cm &= cm - 1;
        const uint32_t rj = __shfl_sync(kFull, row, j);
        const uint64_t lj = __shfl_sync(kFull, len, j);
        const uint64_t sj = __shfl_sync(kFull, start, j);
        const uint64_t rsj = __shfl_sync(kFull, rs, j);
        if (cm) {                                    // the next candidate's S and R bytes, ahead (as the
          const int j2 = __ffs(cm) - 1;              // signature join's probe does for S)
          const uint64_t l2 = __shfl_sync(kFull, len, j2);
          const uint64_t s2 = __shfl_sync(kFull, start, j2);
          const uint64_t r2 = __shfl_sync(kFull, rs, j2);
          const uint64_t o = 32u * (uint64_t)lane;
          if (o < l2) {
            asm volatile("prefetch.global.L1 [%0];" ::"l"(P.arenaS + s2 + o));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(P.arenaR + r2 + o));
          }
        }
        const bool eq = lj < kNarrowLen ? warp_equal(P.arenaR + rsj, P.arenaS + sj, (uint32_t)lj, emask)
                                        : warp_equal_wide(P.arenaR, rsj, P.arenaS, sj, lj);
        if (eq) {
          if (lane == 0) {
            stage.r[np] = rj;
            stage.s[np] = grp * 32 + (uint64_t)j;
          }
          __syncwarp();
          if (++np == (uint32_t)kVStage) {
            flush_stage(stage, np, VP);
            np = 0;
          }
        }
      }
    }
  }
  if (np) flush_stage(stage, np, VP);
}

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------

static thread_local std::string t_err;

static as_status fail(as_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return st;
}

static as_status cuda_fail(cudaError_t e, const char* where) {
  return fail(AS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// The instantiations of the signature kernel: table addressing (AT400),
// components, shape (warps per block, blocks in flight per key) and whether
// it runs over the virtual rows of a batch (4 components only).
static_assert(kLKShapeCount == 3, "one case per shape below");
template <bool AT400, int NCOMP, int SHAPE, bool BATCH>
static cudaError_t key_kernel_attr() {
  constexpr LKShape k = kLKShapes[SHAPE];
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(sig_key_kernel<AT400, NCOMP, k.warps, k.depth, BATCH>),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lk_smem_bytes(k.warps, k.depth));
}
template <bool AT400, int NCOMP, bool BATCH>
static cudaError_t key_kernel_attrs() {
  cudaError_t e = key_kernel_attr<AT400, NCOMP, 0, BATCH>();
  if (e == cudaSuccess) e = key_kernel_attr<AT400, NCOMP, 1, BATCH>();
  if (e == cudaSuccess) e = key_kernel_attr<AT400, NCOMP, 2, BATCH>();
  return e;
}
template <bool AT400, int NCOMP, int SHAPE, bool BATCH>
static void key_kernel_launch(int sms, const uint8_t* arena, const uint64_t* off, uint64_t n, uint64_t* out,
                              const BatchJoin* J, int nj, int s_side, cudaStream_t s) {
  constexpr LKShape k = kLKShapes[SHAPE];
  const uint64_t want = (n + 32ull * k.warps - 1) / (32ull * k.warps);
  const unsigned blocks = (unsigned)(want < (uint64_t)sms ? (want < 1 ? 1 : want) : (uint64_t)sms);
  sig_key_kernel<AT400, NCOMP, k.warps, k.depth, BATCH>
      <<<blocks, 32 * k.warps, lk_smem_bytes(k.warps, k.depth), s>>>(arena, off, n, out, J, nj, s_side);
}
template <bool AT400, int NCOMP, bool BATCH>
static void key_kernel_launch_shape(int shape, int sms, const uint8_t* arena, const uint64_t* off, uint64_t n,
                                    uint64_t* out, const BatchJoin* J, int nj, int s_side, cudaStream_t s) {
  switch (shape) {
    case 1: key_kernel_launch<AT400, NCOMP, 1, BATCH>(sms, arena, off, n, out, J, nj, s_side, s); break;
    case 2: key_kernel_launch<AT400, NCOMP, 2, BATCH>(sms, arena, off, n, out, J, nj, s_side, s); break;
    default: key_kernel_launch<AT400, NCOMP, 0, BATCH>(sms, arena, off, n, out, J, nj, s_side, s); break;
  }
}

constexpr int kSideStreams = 4;
struct DeviceState {
  bool ready = false;
  int sms = 0;
  int verify_blocks_per_sm = 1;
  int prefix_blocks_per_sm = 1;
  int capsig_blocks_per_sm = 1;
  int prefix_thread_blocks_per_sm = 1;
  bool tables_at400 = false;   // dynamic shared memory starts at shared address 0x400
  cudaStream_t side[kSideStreams] = {};   // side streams (SideStream), created with the state
  std::atomic<unsigned> side_next{0};
};

// launch the signature kernel instantiation that matches the device

static std::mutex g_dev_mu;
static DeviceState g_dev[kMaxDevices];

// GF tables by repeated multiplication by x (host), copied to the device once;
// kernel attributes set once per device.
static as_status ensure_device(DeviceState** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(AS_ERR_UNSUPPORTED, "no CUDA device: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(AS_ERR_UNSUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DeviceState& d = g_dev[dev];
  if (!d.ready) {
    static uint16_t h_log[65536], h_alog[65536];
    uint32_t v = 1;
    for (uint32_t i = 0; i < kOrder; i++) {
      h_alog[i] = (uint16_t)v;
      h_log[v] = (uint16_t)i;
      v = gf_times_x(v);
    }
    h_alog[kOrder] = h_alog[0];
    h_log[0] = 0;
    if ((e = cudaMemcpyToSymbol(g_log, h_log, sizeof(h_log))) != cudaSuccess) return cuda_fail(e, "table setup");
    if ((e = cudaMemcpyToSymbol(g_alog, h_alog, sizeof(h_alog))) != cudaSuccess) return cuda_fail(e, "table setup");
    // constant-multiply tables: c_k^(2^s) = x^(k kTile/2 2^s) at (k-1)*kScanLevels+s, then x^-32
    static uint16_t h_const[kConstEntries];
    auto mul = [&](uint32_t a, uint32_t b) -> uint32_t {
      if (a == 0 || b == 0) return 0;
      return h_alog[((uint32_t)h_log[a] + (uint32_t)h_log[b]) % kOrder];
    };
    for (int t = 0; t < kConstCount; t++) {
      uint64_t ex;
      if (t < 4 * kScanLevels) {
        const int k = t / kScanLevels + 1, sh = t % kScanLevels;
        ex = ((uint64_t)k * (kTile / 2) << sh) % kOrder;
      } else {
        ex = kOrder - 32;
      }
      const uint32_t C = h_alog[ex];
      for (uint32_t b = 0; b < 256; b++) {
        h_const[t * 512 + b] = (uint16_t)mul(b, C);
        h_const[t * 512 + 256 + b] = (uint16_t)mul(mul(b, h_alog[8]), C);
      }
    }
    if ((e = cudaMemcpyToSymbol(g_const, h_const, sizeof(h_const))) != cudaSuccess) return cuda_fail(e, "table setup");
    {  // the reduction tables' shared-memory image: row b, word l: T16[b] (l < 32), T24[b] (l >= 32)
      static uint32_t h_red[kRedWords];
      for (uint32_t b = 0; b < 256; b++) {
        uint32_t t16 = b, t24 = b;
        for (int i = 0; i < 16; i++) t16 = gf_times_x(t16);
        for (int i = 0; i < 24; i++) t24 = gf_times_x(t24);
        t16 ^= b << 16;
        t24 ^= b << 24;
        for (int l = 0; l < 64; l++) h_red[b * 64 + l] = l < 32 ? t16 : t24;
      }
      if ((e = cudaMemcpyToSymbol(g_red_img, h_red, sizeof(h_red))) != cudaSuccess) return cuda_fail(e, "table setup");
    }
    // prefix-scan tables: x^(-8 k 2^s) at (k-1)*kPLevels+s
    static uint16_t h_pconst[kPConst * 512];
    for (int t = 0; t < kPConst; t++) {
      const int k = t / kPLevels + 1, sh = t % kPLevels;
      const uint64_t up = ((uint64_t)8 * k << sh) % kOrder;
      const uint32_t C = h_alog[(kOrder - up) % kOrder];
      for (uint32_t b = 0; b < 256; b++) {
        h_pconst[t * 512 + b] = (uint16_t)mul(b, C);
        h_pconst[t * 512 + 256 + b] = (uint16_t)mul(mul(b, h_alog[8]), C);
      }
    }
    if ((e = cudaMemcpyToSymbol(g_pconst, h_pconst, sizeof(h_pconst))) != cudaSuccess) return cuda_fail(e, "table setup");
    if ((e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return cuda_fail(e, "device query");
    {
      if ((e = key_kernel_attrs<true, 4, false>()) != cudaSuccess ||
          (e = key_kernel_attrs<false, 4, false>()) != cudaSuccess ||
          (e = key_kernel_attrs<true, 2, false>()) != cudaSuccess ||
          (e = key_kernel_attrs<false, 2, false>()) != cudaSuccess ||
          (e = key_kernel_attrs<true, 4, true>()) != cudaSuccess ||
          (e = key_kernel_attrs<false, 4, true>()) != cudaSuccess)
        return cuda_fail(e, "kernel attribute");
      {
        constexpr LKShape k = kLKShapes[0];
        const int smem = (int)lk_smem_bytes(k.warps, k.depth, ProbePost::kScratch);
        const int smem_b = (int)lk_smem_bytes(k.warps, k.depth, BuildPost::kScratch);
        if ((e = cudaFuncSetAttribute(
                 reinterpret_cast<const void*>(sig_key_kernel<true, 4, k.warps, k.depth, false, ProbePost>),
                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(
                 reinterpret_cast<const void*>(sig_key_kernel<false, 4, k.warps, k.depth, false, ProbePost>),
                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(
                 reinterpret_cast<const void*>(sig_key_kernel<true, 4, k.warps, k.depth, false, BuildPost>),
                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem_b)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(
                 reinterpret_cast<const void*>(sig_key_kernel<false, 4, k.warps, k.depth, false, BuildPost>),
                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem_b)) != cudaSuccess)
          return cuda_fail(e, "kernel attribute");
      }
    }
    // where dynamic shared memory starts (the tables are its first bytes)
    if ((e = cudaFuncSetAttribute(dyn_smem_base_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemSig)) !=
        cudaSuccess)
      return cuda_fail(e, "kernel attribute");
    dyn_smem_base_kernel<<<1, 32, kSmemSig>>>();
    uint32_t base = 0;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "shared memory probe");
    if ((e = cudaMemcpyFromSymbol(&base, g_dyn_smem_base, sizeof(base))) != cudaSuccess)
      return cuda_fail(e, "shared memory probe");
    d.tables_at400 = base == kTablesAt400;
    for (int i = 0; i < kSideStreams; ++i)
      if ((e = cudaStreamCreateWithFlags(&d.side[i], cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "side stream");
    if ((e = cudaFuncSetAttribute(prefix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemPrefix)) !=
        cudaSuccess)
      return cuda_fail(e, "kernel attribute");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.prefix_blocks_per_sm, prefix_kernel, kPThreads,
                                                           kSmemPrefix)) != cudaSuccess)
      return cuda_fail(e, "occupancy query");
    if (d.prefix_blocks_per_sm < 1) d.prefix_blocks_per_sm = 1;
    if ((e = cudaFuncSetAttribute(capsig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCapSig)) !=
        cudaSuccess)
      return cuda_fail(e, "kernel attribute");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.capsig_blocks_per_sm, capsig_kernel, kCapThreads,
                                                           kSmemCapSig)) != cudaSuccess)
      return cuda_fail(e, "occupancy query");
    if (d.capsig_blocks_per_sm < 1) d.capsig_blocks_per_sm = 1;
    if ((e = cudaFuncSetAttribute(prefix_thread_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSmemCapSig)) != cudaSuccess)
      return cuda_fail(e, "kernel attribute");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.prefix_thread_blocks_per_sm, prefix_thread_kernel,
                                                           kCapThreads, kSmemCapSig)) != cudaSuccess)
      return cuda_fail(e, "occupancy query");
    if (d.prefix_thread_blocks_per_sm < 1) d.prefix_thread_blocks_per_sm = 1;
    if ((e = cudaFuncSetAttribute(sig8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemSig8)) !=
        cudaSuccess)
      return cuda_fail(e, "kernel attribute");
    if ((e = cudaFuncSetAttribute(bl_hash_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBHash)) !=
        cudaSuccess)
      return cuda_fail(e, "kernel attribute");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.verify_blocks_per_sm, verify_kernel<false, true>, kVThreads, 0)) !=
        cudaSuccess)
      return cuda_fail(e, "occupancy query");
    if (d.verify_blocks_per_sm < 1) d.verify_blocks_per_sm = 1;
    d.ready = true;
  }
  *out = &d;
  return AS_OK;
}

// persistent grid: one block per SM, fewer for small inputs (>= ~64 keys per warp)
static unsigned walk_blocks(uint64_t n, int sms) {
  const uint64_t per_block = 64ull * kWarpsPerBlock;
  uint64_t want = (n + per_block - 1) / per_block;
  if (want > (uint64_t)sms) want = (uint64_t)sms;
  return (unsigned)(want < 1 ? 1 : want);
}

static bool misaligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

static uint64_t round256(uint64_t b) { return (b + 255) & ~255ull; }

static bool table_geometry(uint64_t m, float lf, uint64_t* cap, uint32_t* log2cap) {
  if (!(lf > 0.0f && lf <= 1.0f)) return false;
  if (m >= 0xFFFFFFFFull) return false;
  double want = (double)m / (double)lf;
  uint64_t c = 64;
  uint32_t l = 6;
  while ((double)c < want) {
    c <<= 1;
    ++l;
    if (l > 40) return false;
  }
  *cap = c;
  *log2cap = l;
  return true;
}

static as_status launch_sig(const uint8_t* arena, const uint64_t* off, uint64_t n, uint64_t* out, cudaStream_t s,
                            int ncomp = 4, int shape = 0) {
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  if (n == 0) return AS_OK;
  if (shape < 0 || shape >= kLKShapeCount) return fail(AS_ERR_INVALID, "signature kernel shape %d", shape);
  if (ncomp == 2) {
    if (d->tables_at400) key_kernel_launch_shape<true, 2, false>(shape, d->sms, arena, off, n, out, nullptr, 0, 0, s);
    else key_kernel_launch_shape<false, 2, false>(shape, d->sms, arena, off, n, out, nullptr, 0, 0, s);
  } else {
    if (d->tables_at400) key_kernel_launch_shape<true, 4, false>(shape, d->sms, arena, off, n, out, nullptr, 0, 0, s);
    else key_kernel_launch_shape<false, 4, false>(shape, d->sms, arena, off, n, out, nullptr, 0, 0, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "signature kernel launch");
  return AS_OK;
}

// The signatures of one side of a batch over its joins' row ranges (n virtual
// rows; out indexed by virtual row), with the one-key-per-lane kernel.
static as_status launch_sig_batch(const DeviceState* d, const uint8_t* arena, const uint64_t* off, uint64_t n,
                                  uint64_t* out, const BatchJoin* J, int nj, int s_side, int shape, cudaStream_t s) {
  if (n == 0) return AS_OK;
  if (shape < 0 || shape >= kLKShapeCount) return fail(AS_ERR_INVALID, "signature kernel shape %d", shape);
  if (d->tables_at400) key_kernel_launch_shape<true, 4, true>(shape, d->sms, arena, off, n, out, J, nj, s_side, s);
  else key_kernel_launch_shape<false, 4, true>(shape, d->sms, arena, off, n, out, J, nj, s_side, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "batch signature kernel launch");
  return AS_OK;
}

// S relations from this many keys take the fused pass in as_join_probe and as_join
// (measured: 1.5-4 % faster at 1M to 10M keys; for 100k keys as_join's side-stream
// overlap wins)
constexpr uint64_t kFusedProbeFrom = 1ull << 19;

// The whole join's pass over S: the signature kernel (shape 0) with the probe
// of table t fused in (ProbePost; plain inner join).
static as_status launch_sig_probe(const DeviceState* d, const as_table* t, const uint8_t* arenaS,
                                  const uint64_t* offS, const uint32_t* idS, uint64_t n, uint64_t* sigS,
                                  uint32_t* pairs, uint64_t cap_pairs, uint64_t* count, cudaStream_t s) {
  if (n == 0) return AS_OK;
  ProbePost post;
  VerifyParams& P = post.P;
  P.slots = reinterpret_cast<const Slot*>(t->slots);
  P.mask = t->cap - 1;
  P.arenaR = t->arenaR;
  P.offR = t->offR;
  P.idR = t->idR;
  P.arenaS = arenaS;
  P.offS = offS;
  P.idS = idS;
  P.sigS = sigS;
  P.n = n;
  P.pairs = pairs;
  P.cap = cap_pairs;
  P.count = reinterpret_cast<unsigned long long*>(count);
  P.mode = AS_JOIN_INNER;
  P.matched = nullptr;
  P.J = nullptr;
  P.nj = 0;
  P.counts = nullptr;
  P.cap_len = ~0ull;
  post.st = nullptr;
  post.mt = nullptr;
  post.np = 0;
  constexpr LKShape k = kLKShapes[0];
  const uint64_t want = (n + 32ull * k.warps - 1) / (32ull * k.warps);
  const unsigned blocks = (unsigned)(want < (uint64_t)d->sms ? (want < 1 ? 1 : want) : (uint64_t)d->sms);
  const size_t smem = lk_smem_bytes(k.warps, k.depth, ProbePost::kScratch);
  if (d->tables_at400)
    sig_key_kernel<true, 4, k.warps, k.depth, false, ProbePost>
        <<<blocks, 32 * k.warps, smem, s>>>(arenaS, offS, n, sigS, nullptr, 0, 0, post);
  else
    sig_key_kernel<false, 4, k.warps, k.depth, false, ProbePost>
        <<<blocks, 32 * k.warps, smem, s>>>(arenaS, offS, n, sigS, nullptr, 0, 0, post);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "signature and probe kernel launch");
  return AS_OK;
}

// R's signatures with the build fused in (BuildPost): the signature kernel
// (shape 0) inserts each group of keys into the cleared table slots[0..mask].
static as_status launch_sig_build(const DeviceState* d, const uint8_t* arenaR, const uint64_t* offR, uint64_t m,
                                  uint64_t* sigR, Slot* slots, uint64_t mask, uint32_t* flags, cudaStream_t s) {
  if (m == 0) return AS_OK;
  BuildPost post;
  post.slots = slots;
  post.mask = mask;
  post.offR = offR;
  post.flags = flags;
  constexpr LKShape k = kLKShapes[0];
  const uint64_t want = (m + 32ull * k.warps - 1) / (32ull * k.warps);
  const unsigned blocks = (unsigned)(want < (uint64_t)d->sms ? (want < 1 ? 1 : want) : (uint64_t)d->sms);
  const size_t smem = lk_smem_bytes(k.warps, k.depth, BuildPost::kScratch);
  if (d->tables_at400)
    sig_key_kernel<true, 4, k.warps, k.depth, false, BuildPost>
        <<<blocks, 32 * k.warps, smem, s>>>(arenaR, offR, m, sigR, nullptr, 0, 0, post);
  else
    sig_key_kernel<false, 4, k.warps, k.depth, false, BuildPost>
        <<<blocks, 32 * k.warps, smem, s>>>(arenaR, offR, m, sigR, nullptr, 0, 0, post);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "signature and build kernel launch");
  return AS_OK;
}

// Work that may overlap the caller's stream s: fork() makes a side stream
// (from a small per-device pool) wait for everything enqueued on s so far;
// join() makes s wait for everything enqueued on the side stream since.  The
// events are per call, so concurrent callers never wait on each other's
// records; inside CUDA graph capture the fork and the join become edges of
// the graph.
struct SideStream {
  cudaStream_t main = nullptr, side = nullptr;
  bool forked = false;
  as_status fork(DeviceState* d, cudaStream_t s) {
    main = s;
    side = d->side[d->side_next.fetch_add(1u) % kSideStreams];
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "side stream event");
    if ((e = cudaEventRecord(ev, main)) == cudaSuccess) e = cudaStreamWaitEvent(side, ev, 0);
    cudaEventDestroy(ev);                            // released once the device has passed it
    if (e != cudaSuccess) return cuda_fail(e, "side stream fork");
    forked = true;
    return AS_OK;
  }
  as_status join() {
    if (!forked) return AS_OK;
    forked = false;
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "side stream event");
    if ((e = cudaEventRecord(ev, side)) == cudaSuccess) e = cudaStreamWaitEvent(main, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_fail(e, "side stream join");
    return AS_OK;
  }
};

}  // namespace algsig

using namespace algsig;

// NVTX range around each entry point (a profiler shows the library's calls on
// the host timeline; without one attached the calls cost nothing)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

extern "C" {

const char* as_last_error(void) { return t_err.c_str(); }

const char* as_status_string(as_status st) {
  switch (st) {
    case AS_OK: return "AS_OK";
    case AS_ERR_INVALID: return "AS_ERR_INVALID";
    case AS_ERR_NOMEM: return "AS_ERR_NOMEM";
    case AS_ERR_CAPACITY: return "AS_ERR_CAPACITY";
    case AS_ERR_TABLE_FULL: return "AS_ERR_TABLE_FULL";
    case AS_ERR_CUDA: return "AS_ERR_CUDA";
    case AS_ERR_UNSUPPORTED: return "AS_ERR_UNSUPPORTED";
    default: return "AS_ERR_UNKNOWN";
  }
}

int as_version(void) { return 100; }

as_status as_sig_compute(const uint8_t* d_arena, const uint64_t* d_off, uint64_t n, uint64_t* d_sig_out,
                         as_stream stream) {
  NvtxRange nvtx_range("as_sig_compute");
  if (n > 0 && (!d_arena || !d_off || !d_sig_out)) return fail(AS_ERR_INVALID, "as_sig_compute: null pointer");
  if (n > 0 && misaligned16(d_arena)) return fail(AS_ERR_INVALID, "as_sig_compute: arena not 16-byte aligned");
  return launch_sig(d_arena, d_off, n, d_sig_out, (cudaStream_t)stream);
}

as_status as_sig_compute_gf8(const uint8_t* d_arena, const uint64_t* d_off, uint64_t n, uint64_t* d_sig_out,
                             as_stream stream) {
  NvtxRange nvtx_range("as_sig_compute_gf8");
  if (n > 0 && (!d_arena || !d_off || !d_sig_out)) return fail(AS_ERR_INVALID, "as_sig_compute_gf8: null pointer");
  if (n > 0 && misaligned16(d_arena)) return fail(AS_ERR_INVALID, "as_sig_compute_gf8: arena not 16-byte aligned");
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  if (n == 0) return AS_OK;
  const uint64_t want = (n + kG8Threads - 1) / kG8Threads;
  const unsigned blocks = (unsigned)(want < (uint64_t)d->sms * 8 ? want : (uint64_t)d->sms * 8);
  sig8_kernel<<<blocks, kG8Threads, kSmemSig8, (cudaStream_t)stream>>>(d_arena, d_off, n, d_sig_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "byte-symbol signature kernel launch");
  return AS_OK;
}

size_t as_sig_prefix_ws_bytes(uint64_t n) {
  return (size_t)round256(8 * ((n + kPKeysPerBlock - 1) / kPKeysPerBlock + 1));
}

as_status as_sig_prefix_offsets(const uint64_t* d_off, uint64_t n, uint32_t block_bytes, uint64_t* d_pref_off,
                                void* d_ws, size_t ws_bytes, as_stream stream) {
  NvtxRange nvtx_range("as_sig_prefix_offsets");
  if (block_bytes == 0 || block_bytes % 16 != 0)
    return fail(AS_ERR_INVALID, "as_sig_prefix_offsets: block_bytes %u is not a positive multiple of 16", block_bytes);
  if (!d_pref_off || (n > 0 && (!d_off || !d_ws))) return fail(AS_ERR_INVALID, "as_sig_prefix_offsets: null pointer");
  if (n > 0 && ws_bytes < as_sig_prefix_ws_bytes(n))
    return fail(AS_ERR_NOMEM, "as_sig_prefix_offsets: workspace of %zu bytes, %zu needed", ws_bytes,
                as_sig_prefix_ws_bytes(n));
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (n == 0) {
    if ((e = cudaMemsetAsync(d_pref_off, 0, sizeof(uint64_t), s)) != cudaSuccess) return cuda_fail(e, "prefix offsets");
    return AS_OK;
  }
  const uint64_t nblocks = (n + kPKeysPerBlock - 1) / kPKeysPerBlock;
  uint64_t* sums = reinterpret_cast<uint64_t*>(d_ws);
  prefix_count_kernel<<<(unsigned)nblocks, kPThreads, 0, s>>>(d_off, n, block_bytes, d_pref_off, sums);
  prefix_total_kernel<<<1, kPThreads, 0, s>>>(sums, nblocks, d_pref_off, n);
  prefix_offset_kernel<<<(unsigned)nblocks, kPThreads, 0, s>>>(d_pref_off, n, sums);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "prefix offsets launch");
  return AS_OK;
}

as_status as_sig_prefixes(const uint8_t* d_arena, const uint64_t* d_off, uint64_t n, uint32_t block_bytes,
                          const uint64_t* d_pref_off, uint64_t* d_out, as_stream stream) {
  NvtxRange nvtx_range("as_sig_prefixes");
  if (block_bytes == 0 || block_bytes % 16 != 0)
    return fail(AS_ERR_INVALID, "as_sig_prefixes: block_bytes %u is not a positive multiple of 16", block_bytes);
  if (n > 0 && (!d_arena || !d_off || !d_pref_off || !d_out)) return fail(AS_ERR_INVALID, "as_sig_prefixes: null pointer");
  if (n > 0 && misaligned16(d_arena)) return fail(AS_ERR_INVALID, "as_sig_prefixes: arena not 16-byte aligned");
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  if (n == 0) return AS_OK;
  if (block_bytes >= 32) {
    // entries at most every other chunk: one thread per key, the suffix snapshots of prefix_thread_kernel
    const uint64_t want = (n + kCapThreads - 1) / kCapThreads;
    const uint64_t lim = (uint64_t)d->sms * (uint64_t)d->prefix_thread_blocks_per_sm;
    const unsigned blocks = (unsigned)(want < lim ? want : lim);
    prefix_thread_kernel<<<blocks, kCapThreads, kSmemCapSig, (cudaStream_t)stream>>>(d_arena, d_off, n, block_bytes,
                                                                                       d_pref_off, d_out);
  } else {
    // an entry after every chunk: one warp per key, the scan of D over the lanes
    const uint64_t want = (n + kPThreads / 32 - 1) / (kPThreads / 32);
    const uint64_t lim = (uint64_t)d->sms * (uint64_t)d->prefix_blocks_per_sm;   // persistent: one wave
    const unsigned blocks = (unsigned)(want < lim ? want : lim);
    prefix_kernel<<<blocks, kPThreads, kSmemPrefix, (cudaStream_t)stream>>>(d_arena, d_off, n, block_bytes, d_pref_off,
                                                                            d_out);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "prefix kernel launch");
  return AS_OK;
}

as_status as_sig_compute_n(const uint8_t* d_arena, const uint64_t* d_off, uint64_t n, int n_components,
                           uint64_t* d_sig_out, as_stream stream) {
  NvtxRange nvtx_range("as_sig_compute_n");
  if (n_components != 2 && n_components != 4)
    return fail(AS_ERR_INVALID, "as_sig_compute_n: n_components must be 2 or 4 (got %d)", n_components);
  if (n > 0 && (!d_arena || !d_off || !d_sig_out)) return fail(AS_ERR_INVALID, "as_sig_compute_n: null pointer");
  if (n > 0 && misaligned16(d_arena)) return fail(AS_ERR_INVALID, "as_sig_compute_n: arena not 16-byte aligned");
  return launch_sig(d_arena, d_off, n, d_sig_out, (cudaStream_t)stream, n_components);
}

int as_sig_shapes(int* warps, int* depth, int cap) {
  for (int i = 0; i < kLKShapeCount && i < cap; ++i) {
    if (warps) warps[i] = kLKShapes[i].warps;
    if (depth) depth[i] = kLKShapes[i].depth;
  }
  return kLKShapeCount;
}

as_status as_sig_compute_shape(const uint8_t* d_arena, const uint64_t* d_off, uint64_t n, int n_components,
                               int shape, uint64_t* d_sig_out, as_stream stream) {
  NvtxRange nvtx_range("as_sig_compute_shape");
  if (n_components != 2 && n_components != 4)
    return fail(AS_ERR_INVALID, "as_sig_compute_shape: n_components must be 2 or 4 (got %d)", n_components);
  if (shape < 0 || shape >= kLKShapeCount)
    return fail(AS_ERR_INVALID, "as_sig_compute_shape: shape %d outside [0, %d)", shape, kLKShapeCount);
  if (n > 0 && (!d_arena || !d_off || !d_sig_out)) return fail(AS_ERR_INVALID, "as_sig_compute_shape: null pointer");
  if (n > 0 && misaligned16(d_arena)) return fail(AS_ERR_INVALID, "as_sig_compute_shape: arena not 16-byte aligned");
  return launch_sig(d_arena, d_off, n, d_sig_out, (cudaStream_t)stream, n_components, shape);
}

size_t as_join_table_bytes(uint64_t m, float load_factor) {
  uint64_t cap;
  uint32_t l2;
  if (!table_geometry(m, load_factor, &cap, &l2)) return 0;
  return (size_t)(round256(cap * 16) + round256(m * 8) + 256 + round256((m + 31) / 32 * 4));
}

size_t as_join_ws_bytes(uint64_t m, uint64_t n, float load_factor) {
  const size_t t = as_join_table_bytes(m, load_factor);
  return t ? t + 256 + as_join_probe_ws_bytes(n) : 0;
}

as_status as_join_build(void* d_ws, size_t ws_bytes, const uint8_t* d_arenaR, const uint64_t* d_offR,
                        const uint32_t* d_idR, uint64_t m, const uint64_t* d_sigR, float load_factor, as_table* out,
                        as_stream stream) {
  NvtxRange nvtx_range("as_join_build");
  if (!out) return fail(AS_ERR_INVALID, "as_join_build: null table");
  uint64_t cap;
  uint32_t l2;
  if (!table_geometry(m, load_factor, &cap, &l2))
    return fail(AS_ERR_INVALID, "as_join_build: need 0 < load_factor <= 1 and m < 2^32-1");
  if (!d_ws || (m > 0 && (!d_arenaR || !d_offR))) return fail(AS_ERR_INVALID, "as_join_build: null pointer");
  if (m > 0 && misaligned16(d_arenaR)) return fail(AS_ERR_INVALID, "as_join_build: arena not 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(d_ws) & 255u) return fail(AS_ERR_INVALID, "as_join_build: workspace not 256-byte aligned");
  const size_t need = as_join_table_bytes(m, load_factor);
  if (ws_bytes < need)
    return fail(AS_ERR_NOMEM, "as_join_build: workspace of %zu bytes, need %zu", ws_bytes, need);
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t* ws = (uint8_t*)d_ws;
  Slot* slots = (Slot*)ws;
  uint64_t* sig_ws = (uint64_t*)(ws + round256(cap * 16));
  uint32_t* flags = (uint32_t*)(ws + round256(cap * 16) + round256(m * 8));
  cudaError_t e;
  if ((e = cudaMemsetAsync(slots, 0xFF, cap * 16, s)) != cudaSuccess) return cuda_fail(e, "table clear");
  if ((e = cudaMemsetAsync(flags, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "flag clear");
  const uint64_t* sigR = d_sigR;
  if (!sigR && m > 0) {                              // R's signatures with the build in the same kernel
    st = launch_sig_build(d, d_arenaR, d_offR, m, sig_ws, slots, cap - 1, flags, s);
    if (st != AS_OK) return st;
    sigR = sig_ws;
  } else if (m > 0) {
    uint64_t blocks = (m + 255) / 256;
    const uint64_t lim = (uint64_t)d->sms * 16;
    if (blocks > lim) blocks = lim;
    build_kernel<<<(unsigned)blocks, 256, 0, s>>>(slots, cap - 1, sigR, d_offR, m, flags, nullptr, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "build kernel launch");
  }
  out->slots = reinterpret_cast<uint64_t*>(slots);
  out->sigR = sigR ? sigR : sig_ws;
  out->arenaR = d_arenaR;
  out->offR = d_offR;
  out->idR = d_idR;
  out->flags = flags;
  out->m = m;
  out->cap = cap;
  out->log2cap = l2;
  out->reserved = 0;
  out->matched = reinterpret_cast<uint32_t*>(ws + round256(cap * 16) + round256(m * 8) + 256);
  return AS_OK;
}

size_t as_join_probe_ws_bytes(uint64_t n) { return (size_t)(round256(n * 8) + 256); }

// checks shared by the probe entry points
static as_status probe_args(const char* fn, const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS,
                            uint64_t n, uint32_t* d_pairs, uint64_t cap_pairs, uint64_t* d_count) {
  if (!t || !t->slots || !t->flags || !d_count) return fail(AS_ERR_INVALID, "%s: null table or counter", fn);
  if (n > 0 && (!d_arenaS || !d_offS)) return fail(AS_ERR_INVALID, "%s: null relation", fn);
  if (cap_pairs > 0 && !d_pairs) return fail(AS_ERR_INVALID, "%s: null pair buffer", fn);
  if (n > 0 && misaligned16(d_arenaS)) return fail(AS_ERR_INVALID, "%s: arena not 16-byte aligned", fn);
  if (d_pairs && (reinterpret_cast<uintptr_t>(d_pairs) & 7u))
    return fail(AS_ERR_INVALID, "%s: pair buffer not 8-byte aligned", fn);
  return AS_OK;
}

// table walk + verification + compaction of n S keys whose signatures are in sigS
static as_status launch_verify(DeviceState* d, const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS,
                               const uint32_t* d_idS, uint64_t n, const uint64_t* sigS, uint32_t* d_pairs,
                               uint64_t cap_pairs, uint64_t* d_count, cudaStream_t s, int mode = AS_JOIN_INNER,
                               uint64_t cap_len = ~0ull) {
  VerifyParams P;
  P.matched = mode >= AS_JOIN_OUTER_R ? t->matched : nullptr;
  P.cap_len = cap_len;
  P.slots = reinterpret_cast<const Slot*>(t->slots);
  P.mask = t->cap - 1;
  P.arenaR = t->arenaR;
  P.offR = t->offR;
  P.idR = t->idR;
  P.arenaS = d_arenaS;
  P.offS = d_offS;
  P.idS = d_idS;
  P.sigS = sigS;
  P.n = n;
  P.pairs = d_pairs;
  P.cap = cap_pairs;
  P.count = reinterpret_cast<unsigned long long*>(d_count);
  P.mode = mode;
  P.J = nullptr;
  P.nj = 0;
  P.counts = nullptr;
  uint64_t blocks = (n + kVThreads - 1) / kVThreads;
  const uint64_t lim = (uint64_t)d->sms * (uint64_t)d->verify_blocks_per_sm;
  if (blocks > lim) blocks = lim;
  if (mode == AS_JOIN_INNER) verify_kernel<false, true><<<(unsigned)blocks, kVThreads, 0, s>>>(P);
  else verify_kernel<false, false><<<(unsigned)blocks, kVThreads, 0, s>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "probe kernel launch");
  return AS_OK;
}

// optional synchronous count readback and error-flag check
static as_status finish_probe(const char* fn, const as_table* t, uint64_t cap_pairs, uint64_t* d_count,
                              uint64_t* h_count, cudaStream_t s) {
  if (!h_count) return AS_OK;
  uint64_t cnt = 0;
  uint32_t flags = 0;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(&cnt, d_count, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "count readback");
  if ((e = cudaMemcpyAsync(&flags, t->flags, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "flag readback");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "probe");
  *h_count = cnt;
  if (flags & kFlagTableFull) return fail(AS_ERR_TABLE_FULL, "%s: the build could not place every row", fn);
  if (cnt > cap_pairs)
    return fail(AS_ERR_CAPACITY, "%s: %llu pairs, capacity %llu", fn, (unsigned long long)cnt,
                (unsigned long long)cap_pairs);
  return AS_OK;
}

}  // extern "C"

// as_join_probe's work, for it and for as_join_probe_noalloc; fn names the caller in error messages
static as_status probe_impl(const char* fn, const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS,
                            const uint32_t* d_idS, uint64_t n, uint64_t* d_sigS_out, void* d_ws, size_t ws_bytes,
                            uint32_t* d_pairs, uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count,
                            as_stream stream) {
  as_status st = probe_args(fn, t, d_arenaS, d_offS, n, d_pairs, cap_pairs, d_count);
  if (st != AS_OK) return st;
  uint64_t* sigS = d_sigS_out;
  if (!sigS && n > 0) {
    const size_t need = as_join_probe_ws_bytes(n);
    if (!d_ws || ws_bytes < need)
      return fail(AS_ERR_NOMEM, "%s: workspace of %zu bytes, need %zu", fn, d_ws ? ws_bytes : 0, need);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255u) return fail(AS_ERR_INVALID, "%s: workspace not 256-byte aligned", fn);
    sigS = reinterpret_cast<uint64_t*>(d_ws);
  }
  DeviceState* d = nullptr;
  st = ensure_device(&d);
  if (st != AS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(d_count, 0, 8, s)) != cudaSuccess) return cuda_fail(e, "counter clear");
  if (n >= kFusedProbeFrom) {                      // signatures and probe in one kernel
    st = launch_sig_probe(d, t, d_arenaS, d_offS, d_idS, n, sigS, d_pairs, cap_pairs, d_count, s);
    if (st != AS_OK) return st;
  } else if (n > 0) {
    st = launch_sig(d_arenaS, d_offS, n, sigS, s);
    if (st != AS_OK) return st;
    st = launch_verify(d, t, d_arenaS, d_offS, d_idS, n, sigS, d_pairs, cap_pairs, d_count, s);
    if (st != AS_OK) return st;
  }
  return finish_probe(fn, t, cap_pairs, d_count, h_count, s);
}

extern "C" {

as_status as_join_probe(const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS,
                        uint64_t n, uint64_t* d_sigS_out, void* d_ws, size_t ws_bytes, uint32_t* d_pairs,
                        uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count, as_stream stream) {
  NvtxRange nvtx_range("as_join_probe");
  return probe_impl("as_join_probe", t, d_arenaS, d_offS, d_idS, n, d_sigS_out, d_ws, ws_bytes, d_pairs, cap_pairs,
                    d_count, h_count, stream);
}

as_status as_join_probe_sigs(const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS,
                             const uint32_t* d_idS, uint64_t n, const uint64_t* d_sigS, uint32_t* d_pairs,
                             uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count, as_stream stream) {
  NvtxRange nvtx_range("as_join_probe_sigs");
  as_status st = probe_args("as_join_probe_sigs", t, d_arenaS, d_offS, n, d_pairs, cap_pairs, d_count);
  if (st != AS_OK) return st;
  if (n > 0 && !d_sigS) return fail(AS_ERR_INVALID, "as_join_probe_sigs: null signatures");
  DeviceState* d = nullptr;
  st = ensure_device(&d);
  if (st != AS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(d_count, 0, 8, s)) != cudaSuccess) return cuda_fail(e, "counter clear");
  if (n > 0) {
    st = launch_verify(d, t, d_arenaS, d_offS, d_idS, n, d_sigS, d_pairs, cap_pairs, d_count, s);
    if (st != AS_OK) return st;
  }
  return finish_probe("as_join_probe_sigs", t, cap_pairs, d_count, h_count, s);
}

as_status as_join_probe_mode(const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS,
                             const uint32_t* d_idS, uint64_t n, const uint64_t* d_sigS, int mode, uint32_t* d_pairs,
                             uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count, as_stream stream) {
  NvtxRange nvtx_range("as_join_probe_mode");
  as_status st = probe_args("as_join_probe_mode", t, d_arenaS, d_offS, n, d_pairs, cap_pairs, d_count);
  if (st != AS_OK) return st;
  if (mode < AS_JOIN_INNER || mode > AS_JOIN_ANTI_R) return fail(AS_ERR_INVALID, "as_join_probe_mode: mode %d", mode);
  if (n > 0 && !d_sigS) return fail(AS_ERR_INVALID, "as_join_probe_mode: null signatures");
  const bool r_side = mode >= AS_JOIN_OUTER_R;
  if (r_side && t->m > 0 && !t->matched)
    return fail(AS_ERR_INVALID, "as_join_probe_mode: R-side mode %d needs a table from as_join_build (row bitmap)", mode);
  DeviceState* d = nullptr;
  st = ensure_device(&d);
  if (st != AS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(d_count, 0, 8, s)) != cudaSuccess) return cuda_fail(e, "counter clear");
  if (r_side && t->m > 0 && (e = cudaMemsetAsync(t->matched, 0, (t->m + 31) / 32 * 4, s)) != cudaSuccess)
    return cuda_fail(e, "row bitmap clear");
  if (n > 0) {
    st = launch_verify(d, t, d_arenaS, d_offS, d_idS, n, d_sigS, d_pairs, cap_pairs, d_count, s, mode);
    if (st != AS_OK) return st;
  }
  if (r_side && t->m > 0) {                          // the selected R rows after the probe's pairs
    uint64_t blocks = (t->m + 255) / 256;
    const uint64_t lim = (uint64_t)d->sms * 8;
    if (blocks > lim) blocks = lim;
    r_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(t->matched, t->m, mode == AS_JOIN_SEMI_R ? 1u : 0u, t->idR,
                                                   d_pairs, cap_pairs, reinterpret_cast<unsigned long long*>(d_count));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "R-row kernel launch");
  }
  return finish_probe("as_join_probe_mode", t, cap_pairs, d_count, h_count, s);
}

as_status as_join(const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR, uint64_t m,
                  const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint64_t n,
                  float load_factor, void* d_ws, size_t ws_bytes, uint32_t* d_pairs, uint64_t cap_pairs,
                  uint64_t* d_count, uint64_t* h_count, as_stream stream) {
  NvtxRange nvtx_range("as_join");
  const size_t tb = as_join_table_bytes(m, load_factor);
  if (!tb) return fail(AS_ERR_INVALID, "as_join: need 0 < load_factor <= 1 and m < 2^32-1");
  const size_t need = as_join_ws_bytes(m, n, load_factor);
  if (!d_ws || ws_bytes < need) return fail(AS_ERR_NOMEM, "as_join: workspace of %zu bytes, need %zu", ws_bytes, need);
  if (n > 0 && (!d_arenaS || !d_offS)) return fail(AS_ERR_INVALID, "as_join: null relation");
  if (n > 0 && misaligned16(d_arenaS)) return fail(AS_ERR_INVALID, "as_join: arena not 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(d_ws) & 255u) return fail(AS_ERR_INVALID, "as_join: workspace not 256-byte aligned");
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  uint8_t* rest = (uint8_t*)d_ws + tb;
  uint64_t* sigS = reinterpret_cast<uint64_t*>(rest + 256);
  uint64_t* cnt = d_count ? d_count : (uint64_t*)rest;
  cudaStream_t s = (cudaStream_t)stream;
  as_table t;
  if (n >= kFusedProbeFrom) {
    // R's signatures and the build, then S's signatures with the probe fused in (the verification
    // reads the S keys while they may still sit in L2)
    if ((st = as_join_build(d_ws, tb, d_arenaR, d_offR, d_idR, m, nullptr, load_factor, &t, stream)) != AS_OK)
      return st;
    return probe_impl("as_join", &t, d_arenaS, d_offS, d_idS, n, sigS, nullptr, 0, d_pairs, cap_pairs, cnt, h_count,
                      stream);
  }
  // smaller S: its signatures on a side stream, concurrently with R's signatures and the build
  // (kernels of small relations leave SMs idle), then the probe
  SideStream side;
  if (n > 0) {
    if ((st = side.fork(d, s)) != AS_OK) return st;
    if ((st = launch_sig(d_arenaS, d_offS, n, sigS, side.side)) != AS_OK) {
      side.join();
      return st;
    }
  }
  st = as_join_build(d_ws, tb, d_arenaR, d_offR, d_idR, m, nullptr, load_factor, &t, stream);
  const as_status js = side.join();
  if (st != AS_OK) return st;
  if (js != AS_OK) return js;
  return as_join_probe_sigs(&t, d_arenaS, d_offS, d_idS, n, sigS, d_pairs, cap_pairs, cnt, h_count, stream);
}

// ----------------------------------------------------------------------------
// Prefix join: the join on the keys' first L bytes
// ----------------------------------------------------------------------------

size_t as_join_prefix_ws_bytes(uint64_t m, uint64_t n, float load_factor) {
  uint64_t cap;
  uint32_t l2;
  if (!table_geometry(m, load_factor, &cap, &l2)) return 0;
  return (size_t)(round256(cap * 16) + round256(m * 8) + round256(n * 8) + 512);
}

// signatures of the first min(len, L) bytes of every key (one thread per key)
static as_status launch_capped_sigs(DeviceState* d, const uint8_t* arena, const uint64_t* off, uint64_t n, uint64_t L,
                                    uint64_t* out, cudaStream_t s) {
  if (n == 0) return AS_OK;
  const uint64_t want = (n + kCapThreads - 1) / kCapThreads;
  const uint64_t lim = (uint64_t)d->sms * (uint64_t)d->capsig_blocks_per_sm;
  const unsigned blocks = (unsigned)(want < lim ? want : lim);
  capsig_kernel<<<blocks, kCapThreads, kSmemCapSig, s>>>(arena, off, n, L, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? AS_OK : cuda_fail(e, "prefix signature launch");
}

as_status as_join_prefix(const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR, uint64_t m,
                         const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint64_t n,
                         uint64_t prefix_len, float load_factor, void* d_ws, size_t ws_bytes, uint32_t* d_pairs,
                         uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count, as_stream stream) {
  NvtxRange nvtx_range("as_join_prefix");
  uint64_t cap;
  uint32_t l2;
  if (!table_geometry(m, load_factor, &cap, &l2))
    return fail(AS_ERR_INVALID, "as_join_prefix: need 0 < load_factor <= 1 and m < 2^32-1");
  if (prefix_len > kMaxPrefixLen)
    return fail(AS_ERR_INVALID, "as_join_prefix: prefix_len above %llu", (unsigned long long)kMaxPrefixLen);
  if ((m > 0 && (!d_arenaR || !d_offR)) || (n > 0 && (!d_arenaS || !d_offS)) || (cap_pairs > 0 && !d_pairs))
    return fail(AS_ERR_INVALID, "as_join_prefix: null pointer");
  if ((m > 0 && misaligned16(d_arenaR)) || (n > 0 && misaligned16(d_arenaS)))
    return fail(AS_ERR_INVALID, "as_join_prefix: arena not 16-byte aligned");
  if (d_pairs && (reinterpret_cast<uintptr_t>(d_pairs) & 7u))
    return fail(AS_ERR_INVALID, "as_join_prefix: pair buffer not 8-byte aligned");
  const size_t need = as_join_prefix_ws_bytes(m, n, load_factor);
  if (!d_ws || ws_bytes < need)
    return fail(AS_ERR_NOMEM, "as_join_prefix: workspace of %zu bytes, need %zu", ws_bytes, need);
  if (reinterpret_cast<uintptr_t>(d_ws) & 255u) return fail(AS_ERR_INVALID, "as_join_prefix: workspace alignment");
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t* ws = (uint8_t*)d_ws;
  Slot* slots = (Slot*)ws;
  uint64_t* sigR = (uint64_t*)(ws + round256(cap * 16));
  uint64_t* sigS = (uint64_t*)(ws + round256(cap * 16) + round256(m * 8));
  uint8_t* tail = ws + round256(cap * 16) + round256(m * 8) + round256(n * 8);
  uint32_t* flags = (uint32_t*)tail;
  uint64_t* cnt = d_count ? d_count : (uint64_t*)(tail + 256);
  cudaError_t e;
  if ((e = cudaMemsetAsync(slots, 0xFF, cap * 16, s)) != cudaSuccess) return cuda_fail(e, "table clear");
  if ((e = cudaMemsetAsync(flags, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "flag clear");
  if ((e = cudaMemsetAsync(cnt, 0, 8, s)) != cudaSuccess) return cuda_fail(e, "counter clear");
  if ((st = launch_capped_sigs(d, d_arenaR, d_offR, m, prefix_len, sigR, s)) != AS_OK) return st;
  if (m > 0) {
    uint64_t blocks = (m + 255) / 256;
    const uint64_t lim = (uint64_t)d->sms * 16;
    if (blocks > lim) blocks = lim;
    build_kernel<<<(unsigned)blocks, 256, 0, s>>>(slots, cap - 1, sigR, d_offR, m, flags, nullptr, 0, prefix_len);
  }
  if ((st = launch_capped_sigs(d, d_arenaS, d_offS, n, prefix_len, sigS, s)) != AS_OK) return st;
  if (n > 0) {
    as_table t;
    memset(&t, 0, sizeof(t));
    t.slots = reinterpret_cast<uint64_t*>(slots);
    t.sigR = sigR;
    t.arenaR = d_arenaR;
    t.offR = d_offR;
    t.idR = d_idR;
    t.flags = flags;
    t.m = m;
    t.cap = cap;
    t.log2cap = l2;
    if ((st = launch_verify(d, &t, d_arenaS, d_offS, d_idS, n, sigS, d_pairs, cap_pairs, cnt, s, AS_JOIN_INNER,
                            prefix_len)) != AS_OK)
      return st;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "prefix join launch");
  if (h_count) {
    uint64_t c = 0;
    uint32_t flags_h = 0;
    if ((e = cudaMemcpyAsync(&c, cnt, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(e, "count readback");
    if ((e = cudaMemcpyAsync(&flags_h, flags, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return cuda_fail(e, "flag readback");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "prefix join");
    *h_count = c;
    if (flags_h & kFlagTableFull) return fail(AS_ERR_TABLE_FULL, "as_join_prefix: build overflow");
    if (c > cap_pairs)
      return fail(AS_ERR_CAPACITY, "as_join_prefix: %llu pairs, capacity %llu", (unsigned long long)c,
                  (unsigned long long)cap_pairs);
  }
  return AS_OK;
}

// ----------------------------------------------------------------------------
// Radix-partitioned join (partition.cuh)
// ----------------------------------------------------------------------------

static uint32_t part_bits_for(uint64_t m, uint32_t part_bits) {
  if (part_bits != AS_PART_BITS_AUTO) return part_bits;
  uint32_t b = 0;
  while (b < (uint32_t)kPartMaxBits && (m >> (b + 10)) > 0) ++b;   // about 1024 R rows per partition
  return b;
}

// workspace: sigR | sigS | entR | entS | 7 per-partition arrays | slots | flags, counter
static bool part_layout(uint64_t m, uint64_t n, float lf, uint32_t pbits, uint64_t* slots_max, uint64_t* bytes) {
  if (!(lf > 0.0f && lf <= 1.0f) || m >= 0xFFFFFFFFull || n >= 0x100000000ull || pbits > (uint32_t)kPartMaxBits)
    return false;
  const uint64_t P = 1ull << pbits;
  // each partition's table is a power of two >= max(64, rows / lf), so below 2 rows / lf + 64
  const double want = 2.0 * (double)m / (double)lf;
  if (want > (double)(1ull << 40)) return false;                     // the one-table join's limit too
  const uint64_t sm = (uint64_t)want + 64 * P + P;
  *slots_max = sm;
  *bytes = round256(m * 8) + round256(n * 8) + round256(m * 16) + round256(n * 16) + 7 * round256((P + 1) * 8) +
           round256(sm * 16) + 512;
  return true;
}

size_t as_join_part_ws_bytes(uint64_t m, uint64_t n, float load_factor, uint32_t part_bits) {
  uint64_t sm, bytes;
  if (!part_layout(m, n, load_factor, part_bits_for(m, part_bits), &sm, &bytes)) return 0;
  return (size_t)bytes;
}

as_status as_join_partitioned(const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR, uint64_t m,
                              const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint64_t n,
                              float load_factor, uint32_t part_bits, void* d_ws, size_t ws_bytes, uint32_t* d_pairs,
                              uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count, as_stream stream) {
  NvtxRange nvtx_range("as_join_partitioned");
  const uint32_t pbits = part_bits_for(m, part_bits);
  uint64_t smax, need;
  if (!part_layout(m, n, load_factor, pbits, &smax, &need))
    return fail(AS_ERR_INVALID, "as_join_partitioned: need 0 < load_factor <= 1, m < 2^32-1, n < 2^32, part_bits <= %d",
                kPartMaxBits);
  if ((m > 0 && (!d_arenaR || !d_offR)) || (n > 0 && (!d_arenaS || !d_offS)) || (cap_pairs > 0 && !d_pairs))
    return fail(AS_ERR_INVALID, "as_join_partitioned: null pointer");
  if ((m > 0 && misaligned16(d_arenaR)) || (n > 0 && misaligned16(d_arenaS)))
    return fail(AS_ERR_INVALID, "as_join_partitioned: arena not 16-byte aligned");
  if (d_pairs && (reinterpret_cast<uintptr_t>(d_pairs) & 7u))
    return fail(AS_ERR_INVALID, "as_join_partitioned: pair buffer not 8-byte aligned");
  if (!d_ws || ws_bytes < need)
    return fail(AS_ERR_NOMEM, "as_join_partitioned: workspace of %zu bytes, need %llu", ws_bytes,
                (unsigned long long)need);
  if (reinterpret_cast<uintptr_t>(d_ws) & 255u)
    return fail(AS_ERR_INVALID, "as_join_partitioned: workspace not 256-byte aligned");
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t P = 1ull << pbits;
  uint8_t* w = (uint8_t*)d_ws;
  auto take = [&](uint64_t nbytes) { uint8_t* p = w; w += round256(nbytes); return p; };
  uint64_t* sigR = (uint64_t*)take(m * 8);
  uint64_t* sigS = (uint64_t*)take(n * 8);
  PartEntry* entR = (PartEntry*)take(m * 16);
  PartEntry* entS = (PartEntry*)take(n * 16);
  unsigned long long* cntR = (unsigned long long*)take((P + 1) * 8);
  unsigned long long* cntS = (unsigned long long*)take((P + 1) * 8);
  unsigned long long* startR = (unsigned long long*)take((P + 1) * 8);
  unsigned long long* startS = (unsigned long long*)take((P + 1) * 8);
  unsigned long long* curR = (unsigned long long*)take((P + 1) * 8);
  unsigned long long* curS = (unsigned long long*)take((P + 1) * 8);
  unsigned long long* slot_off = (unsigned long long*)take((P + 1) * 8);
  Slot* slots = (Slot*)take(smax * 16);
  uint32_t* flags = (uint32_t*)w;
  uint64_t* cnt = d_count ? d_count : (uint64_t*)(w + 256);
  cudaError_t e;
  if ((e = cudaMemsetAsync(cntR, 0, (P + 1) * 8, s)) != cudaSuccess) return cuda_fail(e, "partition counts");
  if ((e = cudaMemsetAsync(cntS, 0, (P + 1) * 8, s)) != cudaSuccess) return cuda_fail(e, "partition counts");
  if ((e = cudaMemsetAsync(slots, 0xFF, smax * 16, s)) != cudaSuccess) return cuda_fail(e, "table clear");
  if ((e = cudaMemsetAsync(flags, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "flag clear");
  if ((e = cudaMemsetAsync(cnt, 0, 8, s)) != cudaSuccess) return cuda_fail(e, "counter clear");
  if ((st = launch_sig(d_arenaR, d_offR, m, sigR, s)) != AS_OK) return st;
  if ((st = launch_sig(d_arenaS, d_offS, n, sigS, s)) != AS_OK) return st;
  const unsigned gb = (unsigned)d->sms * 4;
  if (m > 0) part_hist_kernel<<<gb, kPartThreads, 0, s>>>(sigR, d_offR, m, pbits, cntR);
  if (n > 0) part_hist_kernel<<<gb, kPartThreads, 0, s>>>(sigS, d_offS, n, pbits, cntS);
  part_layout_kernel<<<1, 1024, 0, s>>>(cntR, cntS, pbits, load_factor, startR, startS, curR, curS, slot_off);
  if (m > 0) part_scatter_kernel<<<gb, kPartThreads, 0, s>>>(sigR, d_offR, m, pbits, curR, entR);
  if (n > 0) part_scatter_kernel<<<gb, kPartThreads, 0, s>>>(sigS, d_offS, n, pbits, curS, entS);
  if (m > 0) part_build_kernel<<<gb, kPartThreads, 0, s>>>(entR, m, pbits, slot_off, slots, flags);
  if (n > 0) {
    PartProbeParams Q;
    Q.entS = entS;
    Q.n = n;
    Q.pbits = pbits;
    Q.slot_off = slot_off;
    Q.slots = slots;
    VerifyParams& V = Q.V;
    memset(&V, 0, sizeof(V));
    V.cap_len = ~0ull;
    V.arenaR = d_arenaR;
    V.offR = d_offR;
    V.idR = d_idR;
    V.arenaS = d_arenaS;
    V.offS = d_offS;
    V.idS = d_idS;
    V.pairs = d_pairs;
    V.cap = cap_pairs;
    V.count = reinterpret_cast<unsigned long long*>(cnt);
    V.mode = AS_JOIN_INNER;
    uint64_t blocks = (n + kVThreads - 1) / kVThreads;
    const uint64_t lim = (uint64_t)d->sms * (uint64_t)d->verify_blocks_per_sm;
    if (blocks > lim) blocks = lim;
    part_probe_kernel<<<(unsigned)blocks, kVThreads, 0, s>>>(Q);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "partitioned join launch");
  if (h_count) {
    uint64_t c = 0;
    uint32_t flags_h = 0;
    if ((e = cudaMemcpyAsync(&c, cnt, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(e, "count readback");
    if ((e = cudaMemcpyAsync(&flags_h, flags, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return cuda_fail(e, "flag readback");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "partitioned join");
    *h_count = c;
    if (flags_h & kFlagTableFull) return fail(AS_ERR_TABLE_FULL, "as_join_partitioned: build overflow");
    if (c > cap_pairs)
      return fail(AS_ERR_CAPACITY, "as_join_partitioned: %llu pairs, capacity %llu", (unsigned long long)c,
                  (unsigned long long)cap_pairs);
  }
  return AS_OK;
}

// ----------------------------------------------------------------------------
// Batches of independent joins
// ----------------------------------------------------------------------------

static_assert(sizeof(BatchJoin) == 96, "BatchJoin layout");

// layout of a batch workspace: descriptors (n_joins + 1) | slots | sigR | sigS | flags
static bool batch_layout(const as_join_desc* descs, int nj, uint64_t mR, uint64_t nS, float lf,
                         uint64_t* slots_total, uint64_t* vr, uint64_t* vs, uint64_t* bytes) {
  if (nj < 1 || !descs || !(lf > 0.0f && lf <= 1.0f) || mR >= 0xFFFFFFFFull) return false;
  uint64_t tot = 0, prev_r = 0, prev_s = 0, sr = 0, ss = 0;
  for (int j = 0; j < nj; j++) {
    const as_join_desc& d = descs[j];
    if (d.r_begin > d.r_end || d.s_begin > d.s_end || d.r_end > mR || d.s_end > nS) return false;
    if (d.r_begin < prev_r || d.s_begin < prev_s) return false;     // ordered, not overlapping
    prev_r = d.r_end;
    prev_s = d.s_end;
    uint64_t cap;
    uint32_t l2;
    if (!table_geometry(d.r_end - d.r_begin, lf, &cap, &l2)) return false;
    tot += cap;
    sr += d.r_end - d.r_begin;
    ss += d.s_end - d.s_begin;
  }
  *slots_total = tot;
  *vr = sr;
  *vs = ss;
  *bytes = round256((uint64_t)(nj + 1) * sizeof(BatchJoin)) + round256(tot * 16) + round256(sr * 8) +
           round256(ss * 8) + 256;
  return true;
}

size_t as_baseline_ws_bytes(uint64_t m, uint64_t n, float load_factor) {
  uint64_t cap;
  uint32_t l2;
  if (!table_geometry(m, load_factor, &cap, &l2)) return 0;
  return (size_t)(round256(cap * 8) + round256(m * 8) + round256(n * 8) + 512);
}

as_status as_baseline_join(const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR, uint64_t m,
                           const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint64_t n,
                           float load_factor, int tagged, void* d_ws, size_t ws_bytes, uint32_t* d_pairs,
                           uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count, as_stream stream) {
  NvtxRange nvtx_range("as_baseline_join");
  uint64_t cap;
  uint32_t l2;
  if (!table_geometry(m, load_factor, &cap, &l2))
    return fail(AS_ERR_INVALID, "as_baseline_join: need 0 < load_factor <= 1 and m < 2^32-1");
  if ((m > 0 && (!d_arenaR || !d_offR)) || (n > 0 && (!d_arenaS || !d_offS)) || (cap_pairs > 0 && !d_pairs))
    return fail(AS_ERR_INVALID, "as_baseline_join: null pointer");
  if ((m > 0 && misaligned16(d_arenaR)) || (n > 0 && misaligned16(d_arenaS)))
    return fail(AS_ERR_INVALID, "as_baseline_join: arena not 16-byte aligned");
  if (d_pairs && (reinterpret_cast<uintptr_t>(d_pairs) & 7u))
    return fail(AS_ERR_INVALID, "as_baseline_join: pair buffer not 8-byte aligned");
  const size_t need = as_baseline_ws_bytes(m, n, load_factor);
  if (!d_ws || ws_bytes < need)
    return fail(AS_ERR_NOMEM, "as_baseline_join: workspace of %zu bytes, need %zu", ws_bytes, need);
  if (reinterpret_cast<uintptr_t>(d_ws) & 255u)
    return fail(AS_ERR_INVALID, "as_baseline_join: workspace not 256-byte aligned");
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t* ws = (uint8_t*)d_ws;
  uint64_t* slots = (uint64_t*)ws;
  uint64_t* hR = (uint64_t*)(ws + round256(cap * 8));
  uint64_t* hS = (uint64_t*)(ws + round256(cap * 8) + round256(m * 8));
  uint8_t* tail = ws + round256(cap * 8) + round256(m * 8) + round256(n * 8);
  uint32_t* flags = (uint32_t*)tail;
  uint64_t* cnt = d_count ? d_count : (uint64_t*)(tail + 256);
  cudaError_t e;
  if ((e = cudaMemsetAsync(slots, 0xFF, cap * 8, s)) != cudaSuccess) return cuda_fail(e, "table clear");
  if ((e = cudaMemsetAsync(flags, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "flag clear");
  if ((e = cudaMemsetAsync(cnt, 0, 8, s)) != cudaSuccess) return cuda_fail(e, "counter clear");
  // S's hashes on a side stream, concurrently with R's hashes and the build (as in as_join)
  SideStream side;
  if (n > 0) {
    if ((st = side.fork(d, s)) != AS_OK) return st;
    bl_hash_kernel<<<walk_blocks(n, d->sms), kThreads, kSmemBHash, side.side>>>(d_arenaS, d_offS, n, hS);
  }
  if (m > 0) {
    bl_hash_kernel<<<walk_blocks(m, d->sms), kThreads, kSmemBHash, s>>>(d_arenaR, d_offR, m, hR);
    uint64_t blocks = (m + 255) / 256;
    const uint64_t lim = (uint64_t)d->sms * 16;
    if (blocks > lim) blocks = lim;
    bl_build_kernel<<<(unsigned)blocks, 256, 0, s>>>(slots, cap - 1, hR, m, tagged, flags);
  }
  const as_status js = side.join();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "baseline hash / build launch");
  if (js != AS_OK) return js;
  if (n > 0) {
    BVerifyParams P;
    P.slots = slots;
    P.mask = cap - 1;
    P.tagged = tagged;
    P.arenaR = d_arenaR;
    P.offR = d_offR;
    P.idR = d_idR;
    P.arenaS = d_arenaS;
    P.offS = d_offS;
    P.idS = d_idS;
    P.hashS = hS;
    P.n = n;
    P.pairs = d_pairs;
    P.cap = cap_pairs;
    P.count = reinterpret_cast<unsigned long long*>(cnt);
    uint64_t blocks = (n + kVThreads - 1) / kVThreads;
    const uint64_t lim = (uint64_t)d->sms * (uint64_t)d->verify_blocks_per_sm;
    if (blocks > lim) blocks = lim;
    bl_verify_kernel<<<(unsigned)blocks, kVThreads, 0, s>>>(P);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "baseline probe launch");
  }
  if (h_count) {
    uint64_t c = 0;
    uint32_t flags_h = 0;
    if ((e = cudaMemcpyAsync(&c, cnt, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(e, "count readback");
    if ((e = cudaMemcpyAsync(&flags_h, flags, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return cuda_fail(e, "flag readback");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "baseline join");
    *h_count = c;
    if (flags_h & kFlagTableFull) return fail(AS_ERR_TABLE_FULL, "as_baseline_join: build overflow");
    if (c > cap_pairs)
      return fail(AS_ERR_CAPACITY, "as_baseline_join: %llu pairs, capacity %llu", (unsigned long long)c,
                  (unsigned long long)cap_pairs);
  }
  return AS_OK;
}

size_t as_join_batch_ws_bytes(const as_join_desc* descs, int n_joins, uint64_t mR, uint64_t nS, float load_factor) {
  uint64_t tot, vr, vs, bytes;
  if (!batch_layout(descs, n_joins, mR, nS, load_factor, &tot, &vr, &vs, &bytes)) return 0;
  return (size_t)bytes;
}

as_status as_join_batch_prepare(const as_join_desc* descs, int n_joins, uint64_t mR, uint64_t nS, float load_factor,
                                void* d_ws, size_t ws_bytes, as_batch* out, as_stream stream) {
  NvtxRange nvtx_range("as_join_batch_prepare");
  if (!out) return fail(AS_ERR_INVALID, "as_join_batch_prepare: null batch");
  uint64_t tot, vr, vs, bytes;
  if (!batch_layout(descs, n_joins, mR, nS, load_factor, &tot, &vr, &vs, &bytes))
    return fail(AS_ERR_INVALID, "as_join_batch_prepare: bad descriptors or load factor");
  if (!d_ws || ws_bytes < bytes)
    return fail(AS_ERR_NOMEM, "as_join_batch_prepare: workspace of %zu bytes, need %llu", ws_bytes,
                (unsigned long long)bytes);
  if (reinterpret_cast<uintptr_t>(d_ws) & 255u) return fail(AS_ERR_INVALID, "as_join_batch_prepare: workspace alignment");
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  std::vector<BatchJoin> h(n_joins + 1);
  uint64_t off = 0, v_r = 0, v_s = 0;
  for (int j = 0; j < n_joins; j++) {
    uint64_t cap;
    uint32_t l2;
    table_geometry(descs[j].r_end - descs[j].r_begin, load_factor, &cap, &l2);
    BatchJoin& b = h[j];
    b.r_begin = descs[j].r_begin;
    b.r_end = descs[j].r_end;
    b.s_begin = descs[j].s_begin;
    b.s_end = descs[j].s_end;
    b.vr = v_r;
    b.vs = v_s;
    b.vbr = b.vbs = 0;
    b.slot_off = off;
    b.mask = cap - 1;
    b.pair_off = descs[j].pair_offset;
    b.pair_cap = descs[j].pair_cap;
    off += cap;
    v_r += b.r_end - b.r_begin;
    v_s += b.s_end - b.s_begin;
  }
  BatchJoin& t = h[n_joins];                       // totals
  memset(&t, 0, sizeof(t));
  t.vr = v_r;
  t.vs = v_s;
  t.r_begin = t.r_end = mR;
  t.s_begin = t.s_end = nS;
  uint8_t* ws = (uint8_t*)d_ws;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(ws, h.data(), sizeof(BatchJoin) * (n_joins + 1), cudaMemcpyHostToDevice,
                           (cudaStream_t)stream)) != cudaSuccess)
    return cuda_fail(e, "batch descriptors");
  if ((e = cudaStreamSynchronize((cudaStream_t)stream)) != cudaSuccess) return cuda_fail(e, "batch descriptors");
  uint64_t o = round256((uint64_t)(n_joins + 1) * sizeof(BatchJoin));
  out->descs = ws;
  out->slots = reinterpret_cast<uint64_t*>(ws + o);
  o += round256(tot * 16);
  out->sigR = reinterpret_cast<uint64_t*>(ws + o);
  o += round256(vr * 8);
  out->sigS = reinterpret_cast<uint64_t*>(ws + o);
  o += round256(vs * 8);
  out->flags = reinterpret_cast<uint32_t*>(ws + o);
  out->n_joins = (uint64_t)n_joins;
  out->slots_total = tot;
  out->mR = vr;
  out->nS = vs;
  // do the joins' rows, in join order, form one ascending run of the relation?
  auto first_of_run = [&](bool s_side) -> uint64_t {
    uint64_t first = 0, next = 0;
    bool any = false;
    for (int j = 0; j < n_joins; j++) {
      const uint64_t b = s_side ? descs[j].s_begin : descs[j].r_begin;
      const uint64_t e = s_side ? descs[j].s_end : descs[j].r_end;
      if (e == b) continue;
      if (!any) { first = b; any = true; }
      else if (b != next) return AS_ROWS_SCATTERED;
      next = e;
    }
    return first;
  };
  out->r_first = first_of_run(false);
  out->s_first = first_of_run(true);
  out->sig_shape = 0;
  out->reserved0 = 0;
  return AS_OK;
}

as_status as_join_batch_run(const as_batch* b, const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR,
                            const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint32_t* d_pairs,
                            uint64_t* d_counts, as_stream stream) {
  NvtxRange nvtx_range("as_join_batch_run");
  if (!b || !b->descs || !d_counts) return fail(AS_ERR_INVALID, "as_join_batch_run: null batch or counters");
  if (!d_arenaR || !d_offR || !d_arenaS || !d_offS) return fail(AS_ERR_INVALID, "as_join_batch_run: null relation");
  if (misaligned16(d_arenaR) || misaligned16(d_arenaS))
    return fail(AS_ERR_INVALID, "as_join_batch_run: arena not 16-byte aligned");
  if (d_pairs && (reinterpret_cast<uintptr_t>(d_pairs) & 7u))
    return fail(AS_ERR_INVALID, "as_join_batch_run: pair buffer not 8-byte aligned");
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  BatchJoin* J = reinterpret_cast<BatchJoin*>(b->descs);
  const int nj = (int)b->n_joins;
  Slot* slots = reinterpret_cast<Slot*>(b->slots);
  if ((e = cudaMemsetAsync(slots, 0xFF, b->slots_total * 16, s)) != cudaSuccess) return cuda_fail(e, "table clear");
  if ((e = cudaMemsetAsync(b->flags, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "flag clear");
  if ((e = cudaMemsetAsync(d_counts, 0, 8 * b->n_joins, s)) != cudaSuccess) return cuda_fail(e, "counter clear");
  batch_bytes_kernel<<<1, 1024, 0, s>>>(J, nj, d_offR, d_offS);
  // S's signatures on a side stream, concurrently with R's signatures and the builds
  SideStream side;
  if (b->nS > 0) {
    if ((st = side.fork(d, s)) != AS_OK) return st;
    if (b->s_first != AS_ROWS_SCATTERED)
      st = launch_sig(d_arenaS, d_offS + b->s_first, b->nS, b->sigS, side.side, 4, b->sig_shape);
    else
      st = launch_sig_batch(d, d_arenaS, d_offS, b->nS, b->sigS, J, nj, 1, b->sig_shape, side.side);
    if (st != AS_OK) {
      side.join();
      return st;
    }
  }
  if (b->mR > 0) {
    if (b->r_first != AS_ROWS_SCATTERED)             // one run of rows: the single-relation kernel
      st = launch_sig(d_arenaR, d_offR + b->r_first, b->mR, b->sigR, s, 4, b->sig_shape);
    else
      st = launch_sig_batch(d, d_arenaR, d_offR, b->mR, b->sigR, J, nj, 0, b->sig_shape, s);
    if (st != AS_OK) {
      side.join();
      return st;
    }
    uint64_t blocks = (b->mR + 255) / 256;
    const uint64_t lim = (uint64_t)d->sms * 16;
    if (blocks > lim) blocks = lim;
    build_kernel<<<(unsigned)blocks, 256, 0, s>>>(slots, 0, b->sigR, d_offR, b->mR, b->flags, J, nj);
  }
  if ((st = side.join()) != AS_OK) return st;
  if (b->nS > 0) {
    VerifyParams P;
    P.slots = slots;
    P.mask = 0;
    P.arenaR = d_arenaR;
    P.offR = d_offR;
    P.idR = d_idR;
    P.arenaS = d_arenaS;
    P.offS = d_offS;
    P.idS = d_idS;
    P.sigS = b->sigS;
    P.n = b->nS;
    P.pairs = d_pairs;
    P.cap = 0;
    P.count = nullptr;
    P.mode = AS_JOIN_INNER;
    P.J = J;
    P.nj = nj;
    P.counts = reinterpret_cast<unsigned long long*>(d_counts);
    uint64_t blocks = (b->nS + kVThreads - 1) / kVThreads;
    const uint64_t lim = (uint64_t)d->sms * (uint64_t)d->verify_blocks_per_sm;
    if (blocks > lim) blocks = lim;
    verify_kernel<true><<<(unsigned)blocks, kVThreads, 0, s>>>(P);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch launch");
  return AS_OK;
}

as_status as_join_batch(const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR, uint64_t mR,
                        const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint64_t nS,
                        const as_join_desc* descs, int n_joins, float load_factor, void* d_ws, size_t ws_bytes,
                        uint32_t* d_pairs, uint64_t* d_counts, as_stream stream) {
  NvtxRange nvtx_range("as_join_batch");
  as_batch b;
  as_status st = as_join_batch_prepare(descs, n_joins, mR, nS, load_factor, d_ws, ws_bytes, &b, stream);
  if (st != AS_OK) return st;
  return as_join_batch_run(&b, d_arenaR, d_offR, d_idR, d_arenaS, d_offS, d_idS, d_pairs, d_counts, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Probe without workspace: S's signatures go to a fixed array in the module's
// device memory instead of a caller workspace, for callers that cannot
// allocate device memory at call time (all of it handed to their own pool, or
// no cudaMalloc/cudaFree allowed on their path since cudaFree synchronises the
// device).  The array is written completely before it is read, so it never
// needs clearing; overlapping calls on one device share it and race.

static __device__ __align__(256) uint64_t g_probe_noalloc_sig[AS_PROBE_NOALLOC_MAX_KEYS];
static void* g_probe_noalloc_addr[algsig::kMaxDevices];   // per device, guarded by g_noalloc_mu
static std::mutex g_noalloc_mu;

extern "C" as_status as_join_probe_noalloc(const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS,
                                           const uint32_t* d_idS, uint64_t n, uint32_t* d_pairs,
                                           uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count,
                                           as_stream stream) {
  NvtxRange nvtx_range("as_join_probe_noalloc");
  using namespace algsig;
  if (n > (uint64_t)AS_PROBE_NOALLOC_MAX_KEYS)
    return fail(AS_ERR_INVALID, "as_join_probe_noalloc: %llu keys, the fixed scratch holds at most %u",
                (unsigned long long)n, (unsigned)AS_PROBE_NOALLOC_MAX_KEYS);
  as_status st = probe_args("as_join_probe_noalloc", t, d_arenaS, d_offS, n, d_pairs, cap_pairs, d_count);
  if (st != AS_OK) return st;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(AS_ERR_UNSUPPORTED, "no CUDA device: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(AS_ERR_UNSUPPORTED, "device index %d out of range", dev);
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_probe_noalloc_addr[dev]) {
      // once per device, with that device current
      if ((e = cudaGetSymbolAddress(&g_probe_noalloc_addr[dev], g_probe_noalloc_sig)) != cudaSuccess) {
        g_probe_noalloc_addr[dev] = nullptr;
        return cuda_fail(e, "scratch address");
      }
    }
    scratch = g_probe_noalloc_addr[dev];
  }
  return probe_impl("as_join_probe_noalloc", t, d_arenaS, d_offS, d_idS, n, static_cast<uint64_t*>(scratch), nullptr,
                    0, d_pairs, cap_pairs, d_count, h_count, stream);
}
