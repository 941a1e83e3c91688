// prefix.cuh -- cumulative (prefix) signatures of every key.
//
// For a key P and a block size B (a multiple of 16 bytes) the cumulative
// signatures are the signatures of its prefixes
//     C_j = sig(P[0 .. min((j+1) B, len))),   j = 0 .. ceil(len / B) - 1
// (one entry, 0, for the empty key).  The last entry is sig(P).  By the
// concatenation rule of Section 3.1 (sig(A || B) = sig(A) + x^(k |A|/2) sig(B)
// for an even byte length |A|), the signature of any substring that starts
// on an even byte a follows from two of them:
//     sig(P[a .. b)) = x^(-k a/2) (sig(P[0 .. b)) + sig(P[0 .. a))).
//
// Kernels.  prefix_count_kernel / prefix_total_kernel / prefix_offset_kernel
// lay out the output: key i's entries start at pref_off[i], an exclusive scan
// of max(1, ceil(len_i / B)).  For B >= 32, prefix_thread_kernel (below)
// computes the entries, one thread per key.  For B = 16 (an entry after every
// chunk) prefix_kernel computes them: one warp per
// key, 512 key bytes per step, lane l taking the key's 16-byte chunk c = 32 s + l
// (realigned to the key's first byte from two aligned chunks, the word part of
// the realignment warp-uniform).  The chunk's value T_c = sum_j q_j x^(k j) is a
// Horner step from zero (gf16.cuh).  With C(c) = sum_{c' <= c} x^(8 k c') T_c'
// the prefix through chunk c, the warp carries D(c) = x^(-8 k c) C(c), which
// obeys D(c) = x^(-8 k) D(c-1) + T_c: an inclusive scan over the lanes whose
// level s multiplies by the constant x^(-8 k 2^s) (tables in shared memory),
// with the previous step's last D entering at lane 0.  Only the lanes whose
// chunk ends a block (or the key) form C = x^(8 k c) D through the log /
// antilog tables and store it.
#pragma once
#include <cstdint>

namespace algsig {

constexpr int kPThreads = 256;          // threads per block of the prefix kernels
constexpr int kPLevels = 5;             // scan levels over 32 lanes
constexpr int kPConst = 4 * kPLevels;   // tables x^(-8 k 2^s), k = 1..4, s = 0..4, at (k-1)*kPLevels+s
// multiply-by-constant tables of the prefix scan (layout of rounds.cuh's), set up once per device
__device__ uint16_t g_pconst[kPConst * 512];

// component-wise multiply of a packed value by x^(-8 k 2^s)
__device__ __forceinline__ uint64_t mul_pscan(const uint16_t* ptab, uint64_t v, int s) {
  uint64_t r = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const uint32_t c = mulc(ptab + (size_t)(k * kPLevels + s) * 512, (uint32_t)(v >> (16 * k)) & 0xFFFFu);
    r |= (uint64_t)c << (16 * k);
  }
  return r;
}
constexpr int kPItems = 4;              // keys per thread in the count / offset kernels
constexpr int kPKeysPerBlock = kPThreads * kPItems;

__device__ __forceinline__ uint64_t prefix_entries(uint64_t len, uint32_t block_bytes) {
  return len == 0 ? 1 : (len + block_bytes - 1) / block_bytes;
}

// block-wide exclusive scan of one value per thread; returns the block total in *total
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* total) {
  __shared__ uint64_t warp_tot[kPThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane >= d) inc += t;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  uint64_t before = 0, all = 0;
  for (int i = 0; i < kPThreads / 32; i++) {
    if (i < w) before += warp_tot[i];
    all += warp_tot[i];
  }
  __syncthreads();
  *total = all;
  return before + inc - v;
}

// pass 1: pref_off[i] = exclusive prefix of the entry counts inside the key's
// block of kPKeysPerBlock keys; block_sums[b] = the block's total
__global__ void __launch_bounds__(kPThreads) prefix_count_kernel(const uint64_t* __restrict__ off, uint64_t n,
                                                                 uint32_t block_bytes, uint64_t* __restrict__ pref_off,
                                                                 uint64_t* __restrict__ block_sums) {
  const uint64_t k0 = (uint64_t)blockIdx.x * kPKeysPerBlock + (uint64_t)threadIdx.x * kPItems;
  uint64_t cnt[kPItems], s = 0;
#pragma unroll
  for (int j = 0; j < kPItems; j++) {
    const uint64_t k = k0 + j;
    cnt[j] = k < n ? prefix_entries(off[k + 1] - off[k], block_bytes) : 0;
    s += cnt[j];
  }
  uint64_t total;
  uint64_t run = block_exclusive_scan(s, &total);
#pragma unroll
  for (int j = 0; j < kPItems; j++) {
    const uint64_t k = k0 + j;
    if (k < n) pref_off[k] = run;
    run += cnt[j];
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// pass 2 (one block): exclusive scan of the block totals in place; pref_off[n] = the total
__global__ void __launch_bounds__(kPThreads) prefix_total_kernel(uint64_t* __restrict__ block_sums, uint64_t nblocks,
                                                                 uint64_t* __restrict__ pref_off, uint64_t n) {
  uint64_t carry = 0;
  for (uint64_t b0 = 0; b0 < nblocks; b0 += kPThreads) {
    const uint64_t b = b0 + threadIdx.x;
    const uint64_t v = b < nblocks ? block_sums[b] : 0;
    uint64_t total;
    const uint64_t ex = block_exclusive_scan(v, &total);
    if (b < nblocks) block_sums[b] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) pref_off[n] = carry;
}

// pass 3: add each block's start
__global__ void __launch_bounds__(kPThreads) prefix_offset_kernel(uint64_t* __restrict__ pref_off, uint64_t n,
                                                                  const uint64_t* __restrict__ block_sums) {
  const uint64_t k0 = (uint64_t)blockIdx.x * kPKeysPerBlock + (uint64_t)threadIdx.x * kPItems;
  const uint64_t add = block_sums[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kPItems; j++)
    if (k0 + j < n) pref_off[k0 + j] += add;
}

// x^(8 k c) T, component-wise, through the log / antilog tables; e1 = 8 c mod 65535
__device__ __forceinline__ uint64_t shift_chunk_value(uint32_t t1, uint32_t t2, uint32_t t3, uint32_t t4, uint32_t e1) {
  uint32_t e = e1;
  uint64_t out = 0;
  const uint32_t t[4] = {t1, t2, t3, t4};
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (t[k]) {
      uint32_t l = (uint32_t)__ldg(&g_log[t[k]]) + e;
      if (l >= kOrder) l -= kOrder;
      out |= (uint64_t)__ldg(&g_alog[l]) << (16 * k);
    }
    e += e1;
    if (e >= kOrder) e -= kOrder;
  }
  return out;
}

// Where lane l's chunk c = 32 s + l stands among the blocks of chunks_per_block
// chunks: block q and place r in it, kept per lane and advanced by 32 chunks per
// step without a division (the lane's start and the per-step advance are
// divided once per kernel).
struct BlockPos {
  uint32_t q, r;              // block index, chunk index inside the block
  uint32_t dq, dr;            // 32 / chunks_per_block, 32 % chunks_per_block
  uint32_t q0, r0;            // lane / chunks_per_block, lane % chunks_per_block
  uint32_t cpb;
  __device__ __forceinline__ void start() { q = q0; r = r0; }
  __device__ __forceinline__ void advance() {
    q += dq;
    r += dr;
    if (r >= cpb) { r -= cpb; q += 1; }
  }
};

// One warp step of a key: lane l's chunk c = c0 + l of the key (realigned to
// the key's first byte from the two aligned chunks ra, rb loaded for it), the
// scan of D over the lanes and the stores of the entries that end in this
// step.  carry: D of the chunk before the step (updated); bp, e1: the lane's
// block position and 8 c mod 65535 (advanced).
template <class Cursor>
__device__ __forceinline__ void prefix_step(const uint4& ra, const uint4& rb, uint32_t a, uint64_t len, uint64_t c0,
                                            BlockPos& bp, uint32_t& e1, uint64_t& carry,
                                            uint64_t* __restrict__ o, const uint4* __restrict__ emask,
                                            const Cursor& rc, const uint16_t* ptab) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t nchunks = (len + 15) / 16;
  const uint64_t c = c0 + lane;
  const uint32_t sh = 8u * (a & 3u);
  uint64_t W = 0;
  if (c < nchunks) {
    uint32_t v0, v1, v2, v3;
    switch (a >> 2) {                              // warp-uniform
      case 0:
        v0 = __funnelshift_r(ra.x, ra.y, sh); v1 = __funnelshift_r(ra.y, ra.z, sh);
        v2 = __funnelshift_r(ra.z, ra.w, sh); v3 = __funnelshift_r(ra.w, rb.x, sh);
        break;
      case 1:
        v0 = __funnelshift_r(ra.y, ra.z, sh); v1 = __funnelshift_r(ra.z, ra.w, sh);
        v2 = __funnelshift_r(ra.w, rb.x, sh); v3 = __funnelshift_r(rb.x, rb.y, sh);
        break;
      case 2:
        v0 = __funnelshift_r(ra.z, ra.w, sh); v1 = __funnelshift_r(ra.w, rb.x, sh);
        v2 = __funnelshift_r(rb.x, rb.y, sh); v3 = __funnelshift_r(rb.y, rb.z, sh);
        break;
      default:
        v0 = __funnelshift_r(ra.w, rb.x, sh); v1 = __funnelshift_r(rb.x, rb.y, sh);
        v2 = __funnelshift_r(rb.y, rb.z, sh); v3 = __funnelshift_r(rb.z, rb.w, sh);
        break;
    }
    const uint64_t rest = len - 16 * c;           // key bytes from this chunk on
    const uint4 m = emask[rest < 16 ? rest : 16];
    v0 &= m.x; v1 &= m.y; v2 &= m.z; v3 &= m.w;
    uint32_t t1 = 0, t2 = 0, t3 = 0, t4 = 0;
    horner_chunk(v0, v1, v2, v3, t1, t2, t3, t4, rc);
    W = (uint64_t)t1 | ((uint64_t)t2 << 16) | ((uint64_t)t3 << 32) | ((uint64_t)t4 << 48);
  }
  if (c0 != 0) {                                   // x^(-8k) D(c0 - 1) enters at lane 0 (zero on a key's first step)
    const uint64_t cin = mul_pscan(ptab, carry, 0);
    if (lane == 0) W ^= cin;
  }
  // levels for the step's live chunks only (warp-uniform)
  const uint32_t live = nchunks - c0 < 32 ? (uint32_t)(nchunks - c0) : 32u;
#pragma unroll
  for (int s = 0; s < kPLevels; s++) {
    if ((1u << s) >= live) break;
    const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, W, 1u << s);
    if (lane >= (1u << s)) W ^= mul_pscan(ptab, t, s);
  }
  if (c < nchunks && (bp.r + 1 == bp.cpb || c + 1 == nchunks))
    o[bp.q] = shift_chunk_value((uint32_t)W & 0xFFFFu, (uint32_t)(W >> 16) & 0xFFFFu, (uint32_t)(W >> 32) & 0xFFFFu,
                                (uint32_t)(W >> 48), e1);
  carry = __shfl_sync(0xFFFFFFFFu, W, 31);
  bp.advance();
  e1 += 256u;
  if (e1 >= kOrder) e1 -= kOrder;
}

// the two aligned chunks lane l's chunk c0 + l is realigned from (zero past the key)
__device__ __forceinline__ void prefix_load(const uint8_t* __restrict__ arena, uint64_t s0, uint64_t len, uint64_t c0,
                                            uint4& ra, uint4& rb) {
  const uint64_t c = c0 + (threadIdx.x & 31u);
  ra = make_uint4(0, 0, 0, 0);
  rb = ra;
  if (16 * c < len) {
    const uint32_t a = (uint32_t)(s0 & 15u);
    const uint8_t* base = arena + s0 - a;           // aligned; key bytes are [a, a + len) from here
    const uint64_t o16 = 16 * c;
    ra = ld16(base + o16);
    if (o16 + 16 < a + len) rb = ld16(base + o16 + 16);
  }
}

// Warps take keys i = warp, warp + nwarps, ...; the work of a warp is the
// sequence of (key, step) items, and the chunks of the next item (and the
// offsets of the next key) are loaded before the current item is computed, so
// the memory latency of a step overlaps the arithmetic of the one before.
__global__ void __launch_bounds__(kPThreads) prefix_kernel(const uint8_t* __restrict__ arena,
                                                           const uint64_t* __restrict__ off, uint64_t n,
                                                           uint32_t block_bytes,
                                                           const uint64_t* __restrict__ pref_off,
                                                           uint64_t* __restrict__ out) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint4 emask[17];
  uint32_t* red = reinterpret_cast<uint32_t*>(smem);
  uint16_t* ptab = reinterpret_cast<uint16_t*>(smem + kRedBytes + 512 * 4);
  for (int i = threadIdx.x; i < kPConst * 512 / 2; i += blockDim.x)
    reinterpret_cast<uint32_t*>(ptab)[i] = reinterpret_cast<const uint32_t*>(g_pconst)[i];
  fill_emask(emask);
  init_red_tables(red, red + kRedWords);            // ends with __syncthreads()
  const RedCursor rc = red_cursor(red);
  const uint32_t lane = threadIdx.x & 31u;
  BlockPos bp;
  bp.cpb = block_bytes / 16u;
  bp.dq = 32u / bp.cpb;
  bp.dr = 32u % bp.cpb;
  bp.q0 = lane / bp.cpb;
  bp.r0 = lane % bp.cpb;
  const uint64_t nwarps = (uint64_t)gridDim.x * (kPThreads / 32);
  uint64_t i = (uint64_t)blockIdx.x * (kPThreads / 32) + (threadIdx.x >> 5);
  if (i >= n) return;                                // warp-uniform
  // current key and its first step's chunks; the next key's offsets
  uint64_t s0 = off[i], len = off[i + 1] - s0, po = pref_off[i];
  uint64_t in = i + nwarps, s0n = 0, lenn = 0, pon = 0;
  if (in < n) { s0n = off[in]; lenn = off[in + 1] - s0n; pon = pref_off[in]; }
  uint64_t c0 = 0;
  uint4 ra, rb;
  prefix_load(arena, s0, len, 0, ra, rb);
  uint64_t carry = 0;
  uint32_t e1 = 8u * lane;
  bp.start();
  for (;;) {
    // the item after this one: the key's next step, or the next key's first
    const uint64_t nchunks = (len + 15) / 16;
    const bool more = c0 + 32 < nchunks;
    const bool next_key = !more && in < n;
    uint4 ra2 = make_uint4(0, 0, 0, 0), rb2 = ra2;
    if (more) prefix_load(arena, s0, len, c0 + 32, ra2, rb2);
    else if (next_key) prefix_load(arena, s0n, lenn, 0, ra2, rb2);
    uint64_t s0nn = 0, lennn = 0, ponn = 0;
    const uint64_t inn = in + nwarps;
    if (next_key && inn < n) { s0nn = off[inn]; lennn = off[inn + 1] - s0nn; ponn = pref_off[inn]; }
    // this item
    if (len == 0) {
      if (lane == 0) out[po] = 0;
    } else {
      prefix_step(ra, rb, (uint32_t)(s0 & 15u), len, c0, bp, e1, carry, out + po, emask, rc, ptab);
    }
    if (more) {
      c0 += 32;
    } else if (next_key) {
      i = in; s0 = s0n; len = lenn; po = pon;
      in = inn; s0n = s0nn; lenn = lennn; pon = ponn;
      c0 = 0;
      carry = 0;
      e1 = 8u * lane;
      bp.start();
    } else {
      break;
    }
    ra = ra2;
    rb = rb2;
  }
}

// Signatures of the first min(len, cap_len) bytes of every key, one thread per
// key (the prefix join's keys, all about equally long once capped).  A thread
// runs Horner's rule over its key's realigned chunks from the last to the
// first (gf16.cuh's step; the last chunk masked past the key's end, the first
// below its even start lo), then moves the result back by x^-(k lo/2).
constexpr int kCapThreads = 1024;       // threads per block of capsig_kernel (39 registers a thread)

__global__ void __launch_bounds__(kCapThreads) capsig_kernel(const uint8_t* __restrict__ arena,
                                                           const uint64_t* __restrict__ off, uint64_t n,
                                                           uint64_t cap_len, uint64_t* __restrict__ out) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint4 emask[17];
  uint32_t* red = reinterpret_cast<uint32_t*>(smem);
  uint16_t* inv32 = reinterpret_cast<uint16_t*>(smem + kRedBytes + 512 * 4);
  for (int i = threadIdx.x; i < 256; i += blockDim.x)      // the x^-32 table of the tile combination
    reinterpret_cast<uint32_t*>(inv32)[i] = reinterpret_cast<const uint32_t*>(g_const + 4 * kScanLevels * 512)[i];
  fill_emask(emask);
  init_red_tables(red, red + kRedWords);                     // ends with __syncthreads()
  const RedCursor rc = red_cursor(red);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t s0 = off[i];
    uint64_t len = off[i + 1] - s0;
    if (len > cap_len) len = cap_len;
    uint32_t a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    const uint32_t a = (uint32_t)(s0 & 15u), odd = a & 1u, lo = a - odd, sh = 8u * odd;
    if (len > 0) {
      const uint8_t* base = arena + (s0 - a);                // aligned chunk holding the key's first byte
      const uint64_t C = (lo + len + 15) >> 4;               // realigned chunks: bytes [16 c + odd, 16 c + 16 + odd)
      const uint32_t tail_e = (uint32_t)(lo + len - 16 * (C - 1));
      // the odd realignment of chunk c reads the first word of chunk c + 1
      uint32_t nxt0 = (odd && tail_e == 16) ? __ldg(reinterpret_cast<const uint32_t*>(base + 16 * C)) : 0u;
      for (uint64_t c = C; c-- > 0;) {
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(base + 16 * c));
        uint32_t v0 = __funnelshift_r(w.x, w.y, sh), v1 = __funnelshift_r(w.y, w.z, sh);
        uint32_t v2 = __funnelshift_r(w.z, w.w, sh), v3 = __funnelshift_r(w.w, nxt0, sh);
        if (c == C - 1) {
          const uint4 m = emask[tail_e];
          v0 &= m.x; v1 &= m.y; v2 &= m.z; v3 &= m.w;
        }
        if (c == 0) {
          const uint4 m = emask[lo];
          v0 &= ~m.x; v1 &= ~m.y; v2 &= ~m.z; v3 &= ~m.w;
        }
        horner_chunk(v0, v1, v2, v3, a1, a2, a3, a4, rc);
        nxt0 = w.x;
      }
    }
    const uint64_t P = (uint64_t)a1 | ((uint64_t)a2 << 16) | ((uint64_t)a3 << 32) | ((uint64_t)a4 << 48);
    out[i] = lo_correct_inv(inv32, P, lo, rc);
  }
}

// Cumulative signatures, one thread per key.  The thread runs the backward
// Horner rule of capsig_kernel over the key's realigned chunks; since B is a
// multiple of 16 every block boundary b_j = lo + (j+1) B falls at offset lo of
// chunk c_j = (j+1) B/16, and the suffix of the key from b_j is one more Horner
// step at c_j with the bytes below lo masked (acc'_j, relative to the chunk's
// start).  It is parked in out[j]; once the whole signature S is known,
//     C_j = S + x^(8 k c_j - k lo/2) acc'_j
// (prefix = whole key minus suffix, the suffix moved to its place), formed
// through the log / antilog tables, once per stored entry.
__global__ void __launch_bounds__(kCapThreads) prefix_thread_kernel(const uint8_t* __restrict__ arena,
                                                                    const uint64_t* __restrict__ off, uint64_t n,
                                                                    uint32_t block_bytes,
                                                                    const uint64_t* __restrict__ pref_off,
                                                                    uint64_t* __restrict__ out) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint4 emask[17];
  uint32_t* red = reinterpret_cast<uint32_t*>(smem);
  uint16_t* inv32 = reinterpret_cast<uint16_t*>(smem + kRedBytes + 512 * 4);
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    reinterpret_cast<uint32_t*>(inv32)[i] = reinterpret_cast<const uint32_t*>(g_const + 4 * kScanLevels * 512)[i];
  fill_emask(emask);
  init_red_tables(red, red + kRedWords);                     // ends with __syncthreads()
  const RedCursor rc = red_cursor(red);
  const uint64_t cpb = block_bytes / 16u;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t s0 = off[i], len = off[i + 1] - s0;
    uint64_t* o = out + pref_off[i];
    if (len == 0) {
      o[0] = 0;
      continue;
    }
    const uint64_t nb = (len + block_bytes - 1) / block_bytes;
    const uint32_t a = (uint32_t)(s0 & 15u), odd = a & 1u, lo = a - odd, sh = 8u * odd;
    const uint8_t* base = arena + (s0 - a);
    const uint64_t C = (lo + len + 15) >> 4;
    const uint32_t tail_e = (uint32_t)(lo + len - 16 * (C - 1));
    const uint4 mlo = emask[lo];
    uint32_t a1 = 0, a2 = 0, a3 = 0, a4 = 0;
    uint32_t nxt0 = (odd && tail_e == 16) ? __ldg(reinterpret_cast<const uint32_t*>(base + 16 * C)) : 0u;
    for (uint64_t c = C; c-- > 0;) {
      const uint4 w = __ldg(reinterpret_cast<const uint4*>(base + 16 * c));
      uint32_t v0 = __funnelshift_r(w.x, w.y, sh), v1 = __funnelshift_r(w.y, w.z, sh);
      uint32_t v2 = __funnelshift_r(w.z, w.w, sh), v3 = __funnelshift_r(w.w, nxt0, sh);
      if (c == C - 1) {
        const uint4 m = emask[tail_e];
        v0 &= m.x; v1 &= m.y; v2 &= m.z; v3 &= m.w;
      }
      if (c > 0 && c % cpb == 0 && c / cpb <= nb - 1) {      // block boundary c_j, j = c / cpb - 1
        uint32_t b1 = a1, b2 = a2, b3 = a3, b4 = a4;
        horner_chunk(v0 & ~mlo.x, v1 & ~mlo.y, v2 & ~mlo.z, v3 & ~mlo.w, b1, b2, b3, b4, rc);
        o[c / cpb - 1] = (uint64_t)b1 | ((uint64_t)b2 << 16) | ((uint64_t)b3 << 32) | ((uint64_t)b4 << 48);
      }
      if (c == 0) { v0 &= ~mlo.x; v1 &= ~mlo.y; v2 &= ~mlo.z; v3 &= ~mlo.w; }
      horner_chunk(v0, v1, v2, v3, a1, a2, a3, a4, rc);
      nxt0 = w.x;
    }
    const uint64_t S = lo_correct_inv(inv32, (uint64_t)a1 | ((uint64_t)a2 << 16) | ((uint64_t)a3 << 32) |
                                                 ((uint64_t)a4 << 48), lo, rc);
    for (uint64_t j = 0; j + 1 < nb; j++) {
      const uint64_t v = o[j];
      // e1 = 8 c_j - lo/2 (mod 65535), c_j = (j + 1) cpb; component k uses k e1
      const uint32_t e1 = (uint32_t)((8 * ((j + 1) * cpb) + kOrder - lo / 2) % kOrder);
      o[j] = S ^ shift_chunk_value((uint32_t)v & 0xFFFFu, (uint32_t)(v >> 16) & 0xFFFFu, (uint32_t)(v >> 32) & 0xFFFFu,
                                   (uint32_t)(v >> 48), e1);
    }
    o[nb - 1] = S;
  }
}

constexpr size_t kSmemCapSig = (size_t)kRedBytes + 512 * 4 + 512 * 2;

constexpr size_t kSmemPrefix = (size_t)kRedBytes + 512 * 4 + (size_t)kPConst * 512 * 2;

}  // namespace algsig
