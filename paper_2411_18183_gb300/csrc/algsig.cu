// algsig.cu -- sm_103a kernels and C ABI of the algebraic-signature equi-join.
//
// Pipeline of one join T = Join(R, S) (Figure 2 of the paper):
//   1. signatures of R         sig_tiles_kernel          (Section 3.1)
//   2. build H_sign on R       build_kernel              (Figure 2, formula 3)
//   3. probe with S            probe_kernel: S signatures, table walk,
//                              byte-exact verification, warp-aggregated
//                              output compaction         (Figure 2, formulas 4-5)
//
// Work decomposition of the signature stage.  A key is cut into tiles of
// kTile bytes counted from the key's first byte.  A warp owns a contiguous
// range of keys and walks their tiles in rounds of 32 (one tile per lane).
// Each lane computes the signature of its tile relative to the tile start
// (Horner over 16-byte chunks, see gf16.cuh), then shifts it to the tile's
// position in the key by multiplying with x^(k * symbol offset) through
// log / antilog tables.  Tiles of the same key sit in consecutive lanes; a
// segmented XOR reduction gathers them in the key's first lane, and a key
// that continues into the next round carries its partial signature.  Every
// key's signature is thus written by exactly one lane, with no atomics and no
// zero-initialisation.
//
// Alignment.  Keys start at any byte.  A lane reads the 16-byte aligned
// chunks that cover its tile and, for an odd start, funnel-shifts the stream
// by one byte so that symbols sit on 16-bit boundaries.  The remaining even
// offset lo inside the first chunk only moves every symbol up by lo/2 slots;
// it is undone by the same x^(k * offset) multiply (offset - lo/2).
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/algsig.h"
#include "gf16.cuh"

namespace algsig {

constexpr int kTile = 256;           // bytes of key per lane per round
constexpr int kThreads = 256;        // threads per block of the signature / probe kernels
constexpr int kKeysPerTask = 64;     // keys handed to a warp at a time
constexpr uint64_t kEmpty = ~0ull;   // empty hash slot
constexpr uint32_t kFlagTableFull = 1u;
constexpr int kMaxDevices = 64;

// GF(2^16) logarithm / antilogarithm of x, set up once per device.
__device__ uint16_t g_log[65536];
__device__ uint16_t g_alog[65536];

// ----------------------------------------------------------------------------
// Device helpers
// ----------------------------------------------------------------------------

__device__ __forceinline__ uint4 ldg16(const uint4* p) { return __ldg(p); }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// x^(e) * a for a 16-bit residue a and 0 <= e < 65535, through log/antilog.
__device__ __forceinline__ uint32_t gf_shift(uint32_t a, uint32_t e) {
  if (a == 0) return 0;
  uint32_t t = (uint32_t)__ldg(&g_log[a]) + e;
  if (t >= kOrder) t -= kOrder;
  return __ldg(&g_alog[t]);
}

// Signature contribution of one tile: the bytes [tstart, tstart + tlen) of
// the arena, which hold the key's symbols from symbol offset sym_off on.
// Returns sum_k x^(k*sym_off) * sum_i p_(sym_off+i) x^(k*i), packed.
__device__ __forceinline__ uint64_t tile_sig(const uint8_t* __restrict__ arena, uint64_t tstart, uint32_t tlen,
                                             uint64_t sym_off, const uint32_t* __restrict__ redl) {
  if (tlen == 0) return 0;
  const uint32_t a = (uint32_t)(tstart & 15u);
  const uint32_t odd = a & 1u;
  const int lo = (int)(a - odd);              // even start inside the first realigned chunk
  const int end = lo + (int)tlen;             // realigned end position
  const int C = (end + 15) >> 4;              // realigned chunks
  const uint4* base = reinterpret_cast<const uint4*>(arena + (tstart - a));
  const uint32_t sh = odd * 8u;
  uint32_t a1 = 0, a2 = 0, a3 = 0, a4 = 0;
  uint32_t nxt0 = 0;                          // first word of the aligned chunk after the current one
  if (odd && (end & 15) == 0) nxt0 = ldg16(base + C).x;
  int c = C - 1;
  if (c >= 1) {                               // last chunk: clear bytes past the tile end
    const uint4 w = ldg16(base + c);
    const int e = end - 16 * c;
    uint32_t v0 = __funnelshift_r(w.x, w.y, sh) & byte_range_mask(0, e, 0);
    uint32_t v1 = __funnelshift_r(w.y, w.z, sh) & byte_range_mask(0, e, 1);
    uint32_t v2 = __funnelshift_r(w.z, w.w, sh) & byte_range_mask(0, e, 2);
    uint32_t v3 = __funnelshift_r(w.w, nxt0, sh) & byte_range_mask(0, e, 3);
    horner_chunk(v0, v1, v2, v3, a1, a2, a3, a4, redl);
    nxt0 = w.x;
    --c;
  }
  for (; c >= 1; --c) {                       // whole chunks
    const uint4 w = ldg16(base + c);
    const uint32_t v0 = __funnelshift_r(w.x, w.y, sh);
    const uint32_t v1 = __funnelshift_r(w.y, w.z, sh);
    const uint32_t v2 = __funnelshift_r(w.z, w.w, sh);
    const uint32_t v3 = __funnelshift_r(w.w, nxt0, sh);
    horner_chunk(v0, v1, v2, v3, a1, a2, a3, a4, redl);
    nxt0 = w.x;
  }
  {                                           // first chunk: clear bytes before the tile start
    const uint4 w = ldg16(base);
    const int e = end < 16 ? end : 16;
    uint32_t v0 = __funnelshift_r(w.x, w.y, sh) & byte_range_mask(lo, e, 0);
    uint32_t v1 = __funnelshift_r(w.y, w.z, sh) & byte_range_mask(lo, e, 1);
    uint32_t v2 = __funnelshift_r(w.z, w.w, sh) & byte_range_mask(lo, e, 2);
    uint32_t v3 = __funnelshift_r(w.w, nxt0, sh) & byte_range_mask(lo, e, 3);
    horner_chunk(v0, v1, v2, v3, a1, a2, a3, a4, redl);
  }
  // a_k = sum over slots t of q_t x^(k t), slot t = symbol (sym_off + t - lo/2) of the key.
  const uint32_t eb = (uint32_t)((sym_off % kOrder + kOrder - (uint32_t)(lo >> 1)) % kOrder);
  uint32_t e2 = eb * 2u; if (e2 >= kOrder) e2 -= kOrder;
  uint32_t e3 = e2 + eb; if (e3 >= kOrder) e3 -= kOrder;
  uint32_t e4 = e2 * 2u; if (e4 >= kOrder) e4 -= kOrder;
  const uint64_t s1 = gf_shift(a1, eb), s2 = gf_shift(a2, e2), s3 = gf_shift(a3, e3), s4 = gf_shift(a4, e4);
  return s1 | (s2 << 16) | (s3 << 32) | (s4 << 48);
}

// One round of the tile walk of a warp.  State (kc, tc, carry) is warp-uniform.
// On return, lanes with `complete` hold the finished signature of key `key`
// (whose arena start / length are `kstart` / `klen`); the state is advanced.
struct RoundOut {
  bool complete;
  uint64_t key, sig, kstart, klen;
};

__device__ __forceinline__ RoundOut sig_round(const uint8_t* __restrict__ arena, const uint64_t* __restrict__ off,
                                              uint64_t& kc, uint64_t k_end, uint64_t& tc, uint64_t& carry,
                                              const uint32_t* __restrict__ redl) {
  const uint32_t FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const uint64_t kl = kc + (uint64_t)lane;
  uint64_t sl = 0, ll = 0;
  uint32_t rc = 0;                                 // tiles of key-lane left, clamped to 33
  if (kl < k_end) {
    sl = off[kl];
    ll = off[kl + 1] - sl;
    uint64_t nt = ll == 0 ? 1 : (ll + kTile - 1) / kTile;
    if (lane == 0) nt -= tc;
    rc = nt > 33 ? 33u : (uint32_t)nt;
  }
  uint32_t cum = rc;                               // inclusive scan over lanes
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, cum, d);
    if (lane >= d) cum += t;
  }
  const uint32_t total = __shfl_sync(FULL, cum, 31);
  int q = 0;                                       // key-lane of slot `lane`: first q with cum[q] > lane
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const uint32_t cv = __shfl_sync(FULL, cum, q + d - 1);
    if (cv <= (uint32_t)lane) q += d;
  }
  const bool active = (uint32_t)lane < total;
  const uint32_t cq = __shfl_sync(FULL, cum, q);
  const uint32_t rq = __shfl_sync(FULL, rc, q);
  const uint64_t sq = __shfl_sync(FULL, sl, q);
  const uint64_t lq = __shfl_sync(FULL, ll, q);
  const uint32_t slot0 = cq - rq;                  // first slot of key-lane q in this round
  const uint64_t tile = (uint64_t)((uint32_t)lane - slot0) + (q == 0 ? tc : 0);
  uint64_t contrib = 0;
  if (active) {
    const uint64_t toff = tile * (uint64_t)kTile;
    const uint64_t rest = lq > toff ? lq - toff : 0;
    const uint32_t tlen = rest < (uint64_t)kTile ? (uint32_t)rest : (uint32_t)kTile;
    contrib = tile_sig(arena, sq + toff, tlen, toff >> 1, redl);
  }
  // segmented XOR towards the first lane of each key group
  const int g = active ? q : 32 + lane;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t o = __shfl_down_sync(FULL, contrib, d);
    const int og = __shfl_down_sync(FULL, g, d);
    if (lane + d < 32 && og == g) contrib ^= o;
  }
  const bool head = active && (uint32_t)lane == slot0;
  if (head && q == 0) contrib ^= carry;
  RoundOut r;
  r.complete = head && (slot0 + rq <= 32u);
  r.key = kc + (uint64_t)q;
  r.sig = contrib;
  r.kstart = sq;
  r.klen = lq;
  // advance the walk
  if (total <= 32u) {
    const uint64_t loaded = k_end - kc < 32 ? k_end - kc : 32;
    kc += loaded;
    tc = 0;
    carry = 0;
  } else {
    const int q31 = __shfl_sync(FULL, q, 31);
    const uint32_t s31 = __shfl_sync(FULL, slot0, 31);
    const uint32_t c31 = __shfl_sync(FULL, cq, 31);
    const uint64_t part = __shfl_sync(FULL, contrib, (int)s31);
    if (c31 == 32u) {                              // key of slot 31 ends exactly at the round end
      kc += (uint64_t)q31 + 1;
      tc = 0;
      carry = 0;
    } else {
      tc = (q31 == 0 ? tc : 0) + (uint64_t)(32u - s31);
      kc += (uint64_t)q31;
      carry = part;
    }
  }
  return r;
}

// ----------------------------------------------------------------------------
// Signature kernel
// ----------------------------------------------------------------------------

__global__ void __launch_bounds__(kThreads) sig_tiles_kernel(const uint8_t* __restrict__ arena,
                                                             const uint64_t* __restrict__ off, uint64_t n,
                                                             uint64_t* __restrict__ sig_out) {
  extern __shared__ uint32_t smem[];
  init_red_tables(smem, smem + kRedWords);
  const int lane = threadIdx.x & 31;
  const uint32_t* redl = smem + lane;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t ntasks = (n + kKeysPerTask - 1) / kKeysPerTask;
  for (uint64_t task = warp; task < ntasks; task += nwarps) {
    uint64_t kc = task * kKeysPerTask;
    const uint64_t k_end = kc + kKeysPerTask < n ? kc + kKeysPerTask : n;
    uint64_t tc = 0, carry = 0;
    while (kc < k_end) {
      const RoundOut r = sig_round(arena, off, kc, k_end, tc, carry, redl);
      if (r.complete) sig_out[r.key] = r.sig;
    }
  }
}

// ----------------------------------------------------------------------------
// Build: insert every R row into the open-addressing table (linear probing)
// ----------------------------------------------------------------------------

__global__ void build_kernel(uint64_t* __restrict__ slots, uint64_t mask, const uint64_t* __restrict__ sigR,
                             const uint64_t* __restrict__ offR, uint64_t m, uint32_t* __restrict__ flags) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; row < m; row += stride) {
    const uint64_t len = offR[row + 1] - offR[row];
    const uint64_t h = sig_hash(sigR[row], len);
    const uint64_t word = (h & 0xFFFFFFFF00000000ull) | row;
    uint64_t b = h & mask;
    bool placed = false;
    for (uint64_t step = 0; step <= mask; ++step) {
      const uint64_t cur = *(volatile const uint64_t*)(slots + b);
      if (cur == kEmpty) {
        const unsigned long long prev =
            atomicCAS(reinterpret_cast<unsigned long long*>(slots + b), (unsigned long long)kEmpty,
                      (unsigned long long)word);
        if (prev == kEmpty) { placed = true; break; }
      }
      b = (b + 1) & mask;
    }
    if (!placed) atomicOr(flags, kFlagTableFull);
  }
}

// ----------------------------------------------------------------------------
// Probe: S signatures + table walk + verification + compaction
// ----------------------------------------------------------------------------

struct ProbeParams {
  const uint64_t* slots;
  uint64_t mask;
  const uint64_t* sigR;
  const uint8_t* arenaR;
  const uint64_t* offR;
  const uint32_t* idR;
  const uint8_t* arenaS;
  const uint64_t* offS;
  const uint32_t* idS;
  uint64_t n;
  uint64_t* sigS_out;
  uint32_t* pairs;
  uint64_t cap;
  unsigned long long* count;
};

// the `need` (1..8) bytes starting at p, little-endian in the low bytes; reads
// only aligned 8-byte words that hold at least one of them
__device__ __forceinline__ uint64_t ld_bytes8(const uint8_t* p, uint32_t need) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint64_t* q = reinterpret_cast<const uint64_t*>(a & ~(uintptr_t)7);
  const uint32_t o = (uint32_t)(a & 7u);
  uint64_t v = __ldg(q) >> (8 * o);
  if (o != 0 && o + need > 8) v |= __ldg(q + 1) << (64 - 8 * o);
  return v;
}

__device__ bool bytes_equal(const uint8_t* r, const uint8_t* s, uint64_t len) {
  uint64_t i = 0;
  for (; i + 8 <= len; i += 8)
    if (ld_bytes8(r + i, 8) != ld_bytes8(s + i, 8)) return false;
  const uint32_t rest = (uint32_t)(len - i);
  if (rest == 0) return true;
  const uint64_t mk = (1ull << (8 * rest)) - 1ull;
  return ((ld_bytes8(r + i, rest) ^ ld_bytes8(s + i, rest)) & mk) == 0;
}

// Walk the table for the keys whose lanes have `live` set; emit verified pairs.
// Called by the whole warp.
__device__ __forceinline__ void probe_keys(bool live, uint64_t srow, uint64_t sig, uint64_t sstart, uint64_t slen,
                                           const ProbeParams& P) {
  const uint32_t FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  uint64_t b = 0, steps = 0;
  uint32_t fp = 0, sid = 0;
  if (live) {
    if (P.sigS_out) P.sigS_out[srow] = sig;
    const uint64_t h = sig_hash(sig, slen);
    b = h & P.mask;
    fp = (uint32_t)(h >> 32);
    sid = P.idS ? P.idS[srow] : (uint32_t)srow;
  }
  while (__any_sync(FULL, live)) {
    bool hit = false;
    uint32_t rid = 0;
    if (live) {
      const uint64_t v = __ldg(P.slots + b);
      if (v == kEmpty) {
        live = false;
      } else {
        if ((uint32_t)(v >> 32) == fp) {
          const uint32_t row = (uint32_t)v;
          if (__ldg(P.sigR + row) == sig) {
            const uint64_t rs = __ldg(P.offR + row);
            const uint64_t rl = __ldg(P.offR + row + 1) - rs;
            if (rl == slen && bytes_equal(P.arenaR + rs, P.arenaS + sstart, slen)) {
              hit = true;
              rid = P.idR ? __ldg(P.idR + row) : row;
            }
          }
        }
        b = (b + 1) & P.mask;
        if (++steps > P.mask) live = false;
      }
    }
    const uint32_t hm = __ballot_sync(FULL, hit);
    if (hm) {
      const int leader = __ffs(hm) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(P.count, (unsigned long long)__popc(hm));
      base = __shfl_sync(FULL, base, leader);
      if (hit) {
        const unsigned long long idx = base + (unsigned long long)__popc(hm & lanemask_lt());
        if (idx < P.cap) {
          const uint64_t pr = (uint64_t)rid | ((uint64_t)sid << 32);
          reinterpret_cast<uint64_t*>(P.pairs)[idx] = pr;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) probe_kernel(ProbeParams P) {
  extern __shared__ uint32_t smem[];
  init_red_tables(smem, smem + kRedWords);
  const int lane = threadIdx.x & 31;
  const uint32_t* redl = smem + lane;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t ntasks = (P.n + kKeysPerTask - 1) / kKeysPerTask;
  for (uint64_t task = warp; task < ntasks; task += nwarps) {
    uint64_t kc = task * kKeysPerTask;
    const uint64_t k_end = kc + kKeysPerTask < P.n ? kc + kKeysPerTask : P.n;
    uint64_t tc = 0, carry = 0;
    while (kc < k_end) {
      const RoundOut r = sig_round(P.arenaS, P.offS, kc, k_end, tc, carry, redl);
      probe_keys(r.complete, r.key, r.sig, r.kstart, r.klen, P);
    }
  }
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

struct DeviceState {
  bool ready = false;
  int sms = 0;
  int sig_blocks_per_sm = 0;
  int probe_blocks_per_sm = 0;
};

static std::mutex g_dev_mu;
static DeviceState g_dev[kMaxDevices];
constexpr size_t kSigSmem = (size_t)kRedBytes + 512 * 4;

// GF tables by repeated multiplication by x (host), copied to the device once.
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
    if ((e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return cuda_fail(e, "device query");
    if ((e = cudaFuncSetAttribute(sig_tiles_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSigSmem)) !=
        cudaSuccess)
      return cuda_fail(e, "kernel attribute");
    if ((e = cudaFuncSetAttribute(probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSigSmem)) !=
        cudaSuccess)
      return cuda_fail(e, "kernel attribute");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.sig_blocks_per_sm, sig_tiles_kernel, kThreads,
                                                           kSigSmem)) != cudaSuccess)
      return cuda_fail(e, "occupancy query");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.probe_blocks_per_sm, probe_kernel, kThreads,
                                                           kSigSmem)) != cudaSuccess)
      return cuda_fail(e, "occupancy query");
    if (d.sig_blocks_per_sm < 1) d.sig_blocks_per_sm = 1;
    if (d.probe_blocks_per_sm < 1) d.probe_blocks_per_sm = 1;
    d.ready = true;
  }
  *out = &d;
  return AS_OK;
}

static uint64_t task_blocks(uint64_t n, int per_sm, int sms) {
  const uint64_t ntasks = (n + kKeysPerTask - 1) / kKeysPerTask;
  const uint64_t warps_per_block = kThreads / 32;
  uint64_t want = (ntasks + warps_per_block - 1) / warps_per_block;
  const uint64_t full = (uint64_t)per_sm * (uint64_t)sms;
  if (want > full) want = full;
  return want < 1 ? 1 : want;
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

static as_status launch_sig(const uint8_t* arena, const uint64_t* off, uint64_t n, uint64_t* out, cudaStream_t s) {
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  if (n == 0) return AS_OK;
  const uint64_t blocks = task_blocks(n, d->sig_blocks_per_sm, d->sms);
  sig_tiles_kernel<<<(unsigned)blocks, kThreads, kSigSmem, s>>>(arena, off, n, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "signature kernel launch");
  return AS_OK;
}

}  // namespace algsig

using namespace algsig;

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
  if (n > 0 && (!d_arena || !d_off || !d_sig_out)) return fail(AS_ERR_INVALID, "as_sig_compute: null pointer");
  if (n > 0 && misaligned16(d_arena)) return fail(AS_ERR_INVALID, "as_sig_compute: arena not 16-byte aligned");
  return launch_sig(d_arena, d_off, n, d_sig_out, (cudaStream_t)stream);
}

size_t as_join_table_bytes(uint64_t m, float load_factor) {
  uint64_t cap;
  uint32_t l2;
  if (!table_geometry(m, load_factor, &cap, &l2)) return 0;
  return (size_t)(round256(cap * 8) + round256(m * 8) + 256);
}

size_t as_join_ws_bytes(uint64_t m, float load_factor) {
  const size_t t = as_join_table_bytes(m, load_factor);
  return t ? t + 256 : 0;
}

as_status as_join_build(void* d_ws, size_t ws_bytes, const uint8_t* d_arenaR, const uint64_t* d_offR,
                        const uint32_t* d_idR, uint64_t m, const uint64_t* d_sigR, float load_factor, as_table* out,
                        as_stream stream) {
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
  uint64_t* slots = (uint64_t*)ws;
  uint64_t* sig_ws = (uint64_t*)(ws + round256(cap * 8));
  uint32_t* flags = (uint32_t*)(ws + round256(cap * 8) + round256(m * 8));
  cudaError_t e;
  if ((e = cudaMemsetAsync(slots, 0xFF, cap * 8, s)) != cudaSuccess) return cuda_fail(e, "table clear");
  if ((e = cudaMemsetAsync(flags, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "flag clear");
  const uint64_t* sigR = d_sigR;
  if (!sigR && m > 0) {
    st = launch_sig(d_arenaR, d_offR, m, sig_ws, s);
    if (st != AS_OK) return st;
    sigR = sig_ws;
  }
  if (m > 0) {
    uint64_t blocks = (m + 255) / 256;
    const uint64_t lim = (uint64_t)d->sms * 16;
    if (blocks > lim) blocks = lim;
    build_kernel<<<(unsigned)blocks, 256, 0, s>>>(slots, cap - 1, sigR, d_offR, m, flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "build kernel launch");
  }
  out->slots = slots;
  out->sigR = sigR ? sigR : sig_ws;
  out->arenaR = d_arenaR;
  out->offR = d_offR;
  out->idR = d_idR;
  out->flags = flags;
  out->m = m;
  out->cap = cap;
  out->log2cap = l2;
  out->reserved = 0;
  return AS_OK;
}

as_status as_join_probe(const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS,
                        uint64_t n, uint64_t* d_sigS_out, uint32_t* d_pairs, uint64_t cap_pairs, uint64_t* d_count,
                        uint64_t* h_count, as_stream stream) {
  if (!t || !t->slots || !t->flags || !d_count) return fail(AS_ERR_INVALID, "as_join_probe: null table or counter");
  if (n > 0 && (!d_arenaS || !d_offS)) return fail(AS_ERR_INVALID, "as_join_probe: null relation");
  if (cap_pairs > 0 && !d_pairs) return fail(AS_ERR_INVALID, "as_join_probe: null pair buffer");
  if (n > 0 && misaligned16(d_arenaS)) return fail(AS_ERR_INVALID, "as_join_probe: arena not 16-byte aligned");
  if (d_pairs && (reinterpret_cast<uintptr_t>(d_pairs) & 7u))
    return fail(AS_ERR_INVALID, "as_join_probe: pair buffer not 8-byte aligned");
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(d_count, 0, 8, s)) != cudaSuccess) return cuda_fail(e, "counter clear");
  if (n > 0) {
    ProbeParams P;
    P.slots = t->slots;
    P.mask = t->cap - 1;
    P.sigR = t->sigR;
    P.arenaR = t->arenaR;
    P.offR = t->offR;
    P.idR = t->idR;
    P.arenaS = d_arenaS;
    P.offS = d_offS;
    P.idS = d_idS;
    P.n = n;
    P.sigS_out = d_sigS_out;
    P.pairs = d_pairs;
    P.cap = cap_pairs;
    P.count = reinterpret_cast<unsigned long long*>(d_count);
    const uint64_t blocks = task_blocks(n, d->probe_blocks_per_sm, d->sms);
    probe_kernel<<<(unsigned)blocks, kThreads, kSigSmem, s>>>(P);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "probe kernel launch");
  }
  if (h_count) {
    uint64_t cnt = 0;
    uint32_t flags = 0;
    if ((e = cudaMemcpyAsync(&cnt, d_count, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return cuda_fail(e, "count readback");
    if ((e = cudaMemcpyAsync(&flags, t->flags, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return cuda_fail(e, "flag readback");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "probe");
    *h_count = cnt;
    if (flags & kFlagTableFull) return fail(AS_ERR_TABLE_FULL, "as_join_probe: the build could not place every row");
    if (cnt > cap_pairs)
      return fail(AS_ERR_CAPACITY, "as_join_probe: %llu pairs, capacity %llu", (unsigned long long)cnt,
                  (unsigned long long)cap_pairs);
  }
  return AS_OK;
}

as_status as_join(const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR, uint64_t m,
                  const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint64_t n,
                  float load_factor, void* d_ws, size_t ws_bytes, uint32_t* d_pairs, uint64_t cap_pairs,
                  uint64_t* d_count, uint64_t* h_count, as_stream stream) {
  const size_t tb = as_join_table_bytes(m, load_factor);
  if (!tb) return fail(AS_ERR_INVALID, "as_join: need 0 < load_factor <= 1 and m < 2^32-1");
  if (ws_bytes < tb + 256) return fail(AS_ERR_NOMEM, "as_join: workspace of %zu bytes, need %zu", ws_bytes, tb + 256);
  as_table t;
  as_status st = as_join_build(d_ws, tb, d_arenaR, d_offR, d_idR, m, nullptr, load_factor, &t, stream);
  if (st != AS_OK) return st;
  uint64_t* cnt = d_count ? d_count : (uint64_t*)((uint8_t*)d_ws + tb);
  return as_join_probe(&t, d_arenaS, d_offS, d_idS, n, nullptr, d_pairs, cap_pairs, cnt, h_count, stream);
}

}  // extern "C"
