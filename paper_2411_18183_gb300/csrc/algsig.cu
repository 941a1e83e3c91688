// algsig.cu -- sm_103a kernels and C ABI of the algebraic-signature equi-join.
//
// Pipeline of one join T = Join(R, S) (Figure 2 of the paper):
//   1. signatures of R      sig_kernel     (Section 3.1)
//   2. build H_sign on R    build_kernel   (Figure 2, formula 3)
//   3. probe with S         probe_kernel: S signatures, table walk, byte-exact
//                           verification, output compaction (formulas 4-5)
// The signature work of 1 and 3 is the warp tile walk of rounds.cuh: each
// warp streams its share of the arena through shared memory with cp.async,
// one round (32 tiles of kTile bytes) ahead of the arithmetic.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/algsig.h"
#include "gf16.cuh"

namespace algsig {
// GF(2^16) logarithm / antilogarithm of x, set up once per device.
__device__ uint16_t g_log[65536];
__device__ uint16_t g_alog[65536];
}  // namespace algsig

#include "rounds.cuh"

namespace algsig {

constexpr int kWarpsPerBlock = 16;
constexpr int kThreads = 32 * kWarpsPerBlock;   // one block per SM
constexpr int kPairBuf = 64;                    // verified pairs staged per warp before one atomic
constexpr uint64_t kEmpty = ~0ull;              // empty hash slot
constexpr uint32_t kFlagTableFull = 1u;
constexpr int kMaxDevices = 64;

// shared memory: reduction tables | their scratch | per-warp double buffers | per-warp pair buffers
constexpr size_t kSmemTables = (size_t)kRedBytes + 512 * 4;
constexpr size_t kSmemBufs = (size_t)kWarpsPerBlock * 2 * kBufBytes;
constexpr size_t kSmemSig = kSmemTables + kSmemBufs;
constexpr size_t kSmemProbe = kSmemSig + (size_t)kWarpsPerBlock * kPairBuf * 8;

// ----------------------------------------------------------------------------
// Signature kernel
// ----------------------------------------------------------------------------

__global__ void __launch_bounds__(kThreads, 1) sig_kernel(const uint8_t* __restrict__ arena,
                                                          const uint64_t* __restrict__ off, uint64_t n,
                                                          uint64_t* __restrict__ sig_out) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* red = reinterpret_cast<uint32_t*>(smem);
  init_red_tables(red, red + kRedWords);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const uint32_t* redl = red + lane;
  uint8_t* bufs = smem + kSmemTables + (size_t)wib * 2 * kBufBytes;
  const uint64_t warp = (uint64_t)blockIdx.x * kWarpsPerBlock + wib;
  const uint64_t nwarps = (uint64_t)gridDim.x * kWarpsPerBlock;
  uint64_t k_lo, k_hi;
  warp_key_range(off, n, warp, nwarps, &k_lo, &k_hi);
  // rounds r and r+1 are in flight before round r is computed
  Plan cur = plan_round(plan_load(off, k_lo, k_hi), k_lo, k_hi, 0);
  issue_span(bufs, arena, cur);
  Plan nxt = plan_round(plan_load(off, cur.kc_next, k_hi), cur.kc_next, k_hi, cur.tc_next);
  issue_span(bufs + kBufBytes, arena, nxt);
  uint64_t carry = 0;
  for (int r = 0; cur.valid; ++r) {
    const PlanLoad ahead = plan_load(off, nxt.kc_next, k_hi);
    cp_async_wait_prev();
    __syncwarp();
    uint8_t* buf = bufs + (r & 1) * kBufBytes;
    uint32_t a1, a2, a3, a4;
    tile_accumulate(buf, cur.span_lo, cur, redl, a1, a2, a3, a4);
    const TileVals tv = tile_logs(cur, a1, a2, a3, a4);
    __syncwarp();                                   // buf is free: refill it with round r+2
    const Plan nn = plan_round(ahead, nxt.kc_next, k_hi, nxt.tc_next);
    issue_span(buf, arena, nn);
    bool complete;
    const uint64_t s = combine_round(cur, tv, carry, complete);
    if (complete) sig_out[cur.kc + (uint64_t)cur.q] = s;
    cur = nxt;
    nxt = nn;
  }
  cp_async_wait_all();
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

// Byte equality of two keys of length len, by the whole warp: lane l compares
// bytes [8l, 8l+8) of each 256-byte step.  r and s are generic addresses
// (global or shared); only aligned 8-byte words holding a key byte are read.
__device__ __forceinline__ bool warp_equal(const uint8_t* r, const uint8_t* s, uint64_t len) {
  const int lane = threadIdx.x & 31;
  const uintptr_t ra = reinterpret_cast<uintptr_t>(r), sa = reinterpret_cast<uintptr_t>(s);
  const uint32_t ro = (uint32_t)(ra & 7u), so = (uint32_t)(sa & 7u);
  const uint64_t* rw = reinterpret_cast<const uint64_t*>(ra - ro);
  const uint64_t* sw = reinterpret_cast<const uint64_t*>(sa - so);
  const uint64_t rend = ro + len, send = so + len;
  for (uint64_t b = 0; b < len; b += 256) {
    const uint64_t wi = (b >> 3) + (uint64_t)lane;
    const uint64_t r0 = 8 * wi < rend ? rw[wi] : 0;
    const uint64_t s0 = 8 * wi < send ? sw[wi] : 0;
    uint64_t r1 = __shfl_down_sync(kFull, r0, 1);
    uint64_t s1 = __shfl_down_sync(kFull, s0, 1);
    if (lane == 31) {
      r1 = 8 * (wi + 1) < rend ? rw[wi + 1] : 0;
      s1 = 8 * (wi + 1) < send ? sw[wi + 1] : 0;
    }
    const uint64_t rv = ro ? (r0 >> (8 * ro)) | (r1 << (64 - 8 * ro)) : r0;
    const uint64_t sv = so ? (s0 >> (8 * so)) | (s1 << (64 - 8 * so)) : s0;
    const uint64_t pos = b + 8 * (uint64_t)lane;
    const uint64_t nv = len > pos ? len - pos : 0;
    const uint64_t mk = nv >= 8 ? ~0ull : ((1ull << (8 * nv)) - 1ull);
    if (!__all_sync(kFull, ((rv ^ sv) & mk) == 0)) return false;
  }
  return true;
}

// append the staged pairs of this warp to the output (one atomic per flush)
__device__ __forceinline__ void flush_pairs(uint64_t* stage, uint32_t np, const ProbeParams& P) {
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(P.count, (unsigned long long)np);
  base = __shfl_sync(kFull, base, 0);
  __syncwarp();
  for (uint32_t i = (uint32_t)lane; i < np; i += 32) {
    const unsigned long long idx = base + i;
    if (idx < P.cap) reinterpret_cast<uint64_t*>(P.pairs)[idx] = stage[i];
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kThreads, 1) probe_kernel(ProbeParams P) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* red = reinterpret_cast<uint32_t*>(smem);
  init_red_tables(red, red + kRedWords);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const uint32_t* redl = red + lane;
  uint8_t* bufs = smem + kSmemTables + (size_t)wib * 2 * kBufBytes;
  uint64_t* stage = reinterpret_cast<uint64_t*>(smem + kSmemSig) + (size_t)wib * kPairBuf;
  uint32_t np = 0;                                   // staged pairs (warp-uniform)
  const uint64_t warp = (uint64_t)blockIdx.x * kWarpsPerBlock + wib;
  const uint64_t nwarps = (uint64_t)gridDim.x * kWarpsPerBlock;
  uint64_t k_lo, k_hi;
  warp_key_range(P.offS, P.n, warp, nwarps, &k_lo, &k_hi);
  Plan cur = plan_round(plan_load(P.offS, k_lo, k_hi), k_lo, k_hi, 0);
  issue_span(bufs, P.arenaS, cur);
  Plan nxt = plan_round(plan_load(P.offS, cur.kc_next, k_hi), cur.kc_next, k_hi, cur.tc_next);
  issue_span(bufs + kBufBytes, P.arenaS, nxt);
  uint64_t carry = 0;
  for (int r = 0; cur.valid; ++r) {
    const PlanLoad ahead = plan_load(P.offS, nxt.kc_next, k_hi);
    cp_async_wait_prev();
    __syncwarp();
    uint8_t* buf = bufs + (r & 1) * kBufBytes;
    uint32_t a1, a2, a3, a4;
    tile_accumulate(buf, cur.span_lo, cur, redl, a1, a2, a3, a4);
    const TileVals tv = tile_logs(cur, a1, a2, a3, a4);
    __syncwarp();
    const Plan nn = plan_round(ahead, nxt.kc_next, k_hi, nxt.tc_next);
    issue_span(buf, P.arenaS, nn);
    bool live;
    const uint64_t sig = combine_round(cur, tv, carry, live);
    // table walk of the keys finished in this round (their first lanes)
    const uint64_t srow = cur.kc + (uint64_t)cur.q;
    uint64_t b = 0, steps = 0;
    uint32_t fp = 0;
    if (live) {
      if (P.sigS_out) P.sigS_out[srow] = sig;
      const uint64_t h = sig_hash(sig, cur.klen);
      b = h & P.mask;
      fp = (uint32_t)(h >> 32);
    }
    while (__any_sync(kFull, live)) {
      bool cand = false;
      uint32_t row = 0;
      if (live) {
        const uint64_t v = __ldg(P.slots + b);
        if (v == kEmpty) {
          live = false;
        } else {
          if ((uint32_t)(v >> 32) == fp) {
            row = (uint32_t)v;
            if (__ldg(P.sigR + row) == sig) {
              const uint64_t rs = __ldg(P.offR + row);
              cand = __ldg(P.offR + row + 1) - rs == cur.klen;
            }
          }
          b = (b + 1) & P.mask;
          if (++steps > P.mask) live = false;
        }
      }
      uint32_t cm = __ballot_sync(kFull, cand);
      while (cm) {                                   // verify candidates one by one, whole warp
        const int j = __ffs(cm) - 1;
        cm &= cm - 1;
        const uint32_t rj = __shfl_sync(kFull, row, j);
        const uint64_t len = __shfl_sync(kFull, cur.klen, j);
        const uint64_t sj = __shfl_sync(kFull, cur.kstart, j);
        const uint64_t srj = __shfl_sync(kFull, srow, j);
        if (warp_equal(P.arenaR + __ldg(P.offR + rj), P.arenaS + sj, len)) {
          if (lane == 0) {
            const uint32_t rid = P.idR ? __ldg(P.idR + rj) : rj;
            const uint32_t sid = P.idS ? __ldg(P.idS + srj) : (uint32_t)srj;
            stage[np] = (uint64_t)rid | ((uint64_t)sid << 32);
          }
          if (++np == (uint32_t)kPairBuf) {
            flush_pairs(stage, np, P);
            np = 0;
          }
        }
      }
    }
    cur = nxt;
    nxt = nn;
  }
  cp_async_wait_all();
  if (np) flush_pairs(stage, np, P);
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
};

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
    if ((e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return cuda_fail(e, "device query");
    if ((e = cudaFuncSetAttribute(sig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemSig)) !=
        cudaSuccess)
      return cuda_fail(e, "kernel attribute");
    if ((e = cudaFuncSetAttribute(probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemProbe)) !=
        cudaSuccess)
      return cuda_fail(e, "kernel attribute");
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

static as_status launch_sig(const uint8_t* arena, const uint64_t* off, uint64_t n, uint64_t* out, cudaStream_t s) {
  DeviceState* d = nullptr;
  as_status st = ensure_device(&d);
  if (st != AS_OK) return st;
  if (n == 0) return AS_OK;
  sig_kernel<<<walk_blocks(n, d->sms), kThreads, kSmemSig, s>>>(arena, off, n, out);
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
    probe_kernel<<<walk_blocks(n, d->sms), kThreads, kSmemProbe, s>>>(P);
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
