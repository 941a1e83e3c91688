// partition.cuh -- the radix-partitioned signature join.
//
// The join of Figure 2 with both relations first split into P = 2^p
// partitions by the top p bits of the bucket hash of (signature, length), as in
// the partitioned (Grace) hash join the paper sets its method beside (Sections
// 2 and 4): equal keys have equal signatures and lengths, so they fall in the
// same partition, and every partition is joined on its own with a table sized
// for its R rows.  The bucket inside a partition's table comes from the low
// bits of the same hash.  On the GPU the partitions are not materialised as
// keys: a partition holds 16-byte entries (signature, length | row) of its
// rows, and the probe walks S's entries in partition order, so consecutive
// probes read the same small table.  The byte verification reads the keys
// from the arenas, as the unpartitioned probe does.
//
// Every kernel hashes (signature, min(length, 2^32 - 2)), the length the
// entries and the table slots carry.
//
// Kernels, in launch order (after the signatures of R and S):
//   part_hist_kernel    rows per partition (block-local counts, then global)
//   part_layout_kernel  exclusive scans: entry starts per partition, and the
//                       partitions' table sizes (power of two >= max(64, rows / lf))
//                       and slot offsets
//   part_scatter_kernel entries into partition order (block-aggregated cursors)
//   part_build_kernel   R entries into their partition's table (linear probing)
//   part_probe_kernel   S entries: table walk, byte verification, compaction
#pragma once
#include <cstdint>

namespace algsig {

constexpr int kPartMaxBits = 12;                   // at most 4096 partitions
constexpr int kPartThreads = 256;

struct PartEntry {
  uint64_t sig;
  uint64_t key;      // (len32 << 32) | row
};

__device__ __forceinline__ uint32_t part_of(uint64_t h, uint32_t pbits) {
  return pbits ? (uint32_t)(h >> (64u - pbits)) : 0u;
}

// rows per partition of one relation
__global__ void __launch_bounds__(kPartThreads) part_hist_kernel(const uint64_t* __restrict__ sig,
                                                                 const uint64_t* __restrict__ off, uint64_t n,
                                                                 uint32_t pbits, unsigned long long* __restrict__ cnt) {
  __shared__ uint32_t hist[1 << kPartMaxBits];
  const uint32_t P = 1u << pbits;
  for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    atomicAdd(&hist[part_of(sig_hash(sig[i], len32(off[i + 1] - off[i])), pbits)], 1u);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < P; i += blockDim.x)
    if (hist[i]) atomicAdd(cnt + i, (unsigned long long)hist[i]);
}

// One block.  start{R,S}[p] (exclusive scans of the counts, [P] = total),
// cur{R,S} = the starts (scatter cursors), slot_off[p] (exclusive scan of the
// table sizes, [P] = total slots).
__global__ void __launch_bounds__(1024) part_layout_kernel(const unsigned long long* __restrict__ cntR,
                                                           const unsigned long long* __restrict__ cntS,
                                                           uint32_t pbits, float lf,
                                                           unsigned long long* __restrict__ startR,
                                                           unsigned long long* __restrict__ startS,
                                                           unsigned long long* __restrict__ curR,
                                                           unsigned long long* __restrict__ curS,
                                                           unsigned long long* __restrict__ slot_off) {
  __shared__ unsigned long long part_sum[3][1024];
  const uint32_t P = 1u << pbits;
  const uint32_t per = (P + blockDim.x - 1) / blockDim.x;          // consecutive partitions per thread
  const uint32_t p0 = threadIdx.x * per;
  unsigned long long a = 0, b = 0, c = 0;
  for (uint32_t k = 0; k < per && p0 + k < P; k++) {
    const unsigned long long r = cntR[p0 + k];
    a += r;
    b += cntS[p0 + k];
    unsigned long long cap = 64;
    while ((double)cap * (double)lf < (double)r) cap <<= 1;
    c += cap;
  }
  part_sum[0][threadIdx.x] = a;
  part_sum[1][threadIdx.x] = b;
  part_sum[2][threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x < 3) {                                            // serial scan of the 1024 per-thread sums
    unsigned long long run = 0;
    for (uint32_t t = 0; t < blockDim.x; t++) {
      const unsigned long long v = part_sum[threadIdx.x][t];
      part_sum[threadIdx.x][t] = run;
      run += v;
    }
  }
  __syncthreads();
  a = part_sum[0][threadIdx.x];
  b = part_sum[1][threadIdx.x];
  c = part_sum[2][threadIdx.x];
  for (uint32_t k = 0; k < per && p0 + k < P; k++) {
    const uint32_t p = p0 + k;
    startR[p] = curR[p] = a;
    startS[p] = curS[p] = b;
    slot_off[p] = c;
    const unsigned long long r = cntR[p];
    a += r;
    b += cntS[p];
    unsigned long long cap = 64;
    while ((double)cap * (double)lf < (double)r) cap <<= 1;
    c += cap;
  }
  if (p0 < P && p0 + per >= P) {                                    // the thread holding the last partition
    startR[P] = a;
    startS[P] = b;
    slot_off[P] = c;
  }
}

// Entries of one relation into partition order.  Each block takes a run of
// rows, counts them per partition in shared memory, reserves its range of every
// partition with one global atomic (a partition that many rows share, a Zipf-hot
// key's, then takes one increment per block, not per row), and writes its
// entries through shared-memory cursors.
__global__ void __launch_bounds__(kPartThreads) part_scatter_kernel(const uint64_t* __restrict__ sig,
                                                                    const uint64_t* __restrict__ off, uint64_t n,
                                                                    uint32_t pbits,
                                                                    unsigned long long* __restrict__ cur,
                                                                    PartEntry* __restrict__ ent) {
  __shared__ uint32_t cnt[1 << kPartMaxBits];
  __shared__ uint32_t base[1 << kPartMaxBits];      // entry indices fit 32 bits (n < 2^32)
  const uint32_t P = 1u << pbits;
  const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint64_t r0 = (uint64_t)blockIdx.x * per;
  const uint64_t r1 = r0 + per < n ? r0 + per : n;
  for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  for (uint64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x)
    atomicAdd(&cnt[part_of(sig_hash(sig[i], len32(off[i + 1] - off[i])), pbits)], 1u);
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
    if (cnt[i]) base[i] = (uint32_t)atomicAdd(cur + i, (unsigned long long)cnt[i]);
    cnt[i] = 0;
  }
  __syncthreads();
  for (uint64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const uint64_t s = sig[i];
    const uint64_t len = off[i + 1] - off[i];
    const uint32_t p = part_of(sig_hash(s, len32(len)), pbits);
    PartEntry e;
    e.sig = s;
    e.key = ((uint64_t)len32(len) << 32) | i;
    ent[base[p] + atomicAdd(&cnt[p], 1u)] = e;
  }
}

// R entries into their partition's table
__global__ void part_build_kernel(const PartEntry* __restrict__ ent, uint64_t m, uint32_t pbits,
                                  const unsigned long long* __restrict__ slot_off, Slot* __restrict__ slots,
                                  uint32_t* __restrict__ flags) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const PartEntry e = ent[i];
    const uint64_t h = sig_hash(e.sig, e.key >> 32);
    const uint32_t p = part_of(h, pbits);
    Slot* tab = slots + slot_off[p];
    const uint64_t msk = slot_off[p + 1] - slot_off[p] - 1;
    uint64_t b = h & msk;
    bool placed = false;
    for (uint64_t step = 0; step <= msk; ++step) {
      const uint64_t cur = *(volatile const uint64_t*)(&tab[b].key);
      if (cur == kEmpty) {
        const unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(&tab[b].key),
                                                  (unsigned long long)kEmpty, (unsigned long long)e.key);
        if (prev == kEmpty) {
          tab[b].sig = e.sig;
          placed = true;
          break;
        }
      }
      b = (b + 1) & msk;
    }
    if (!placed) atomicOr(flags, kFlagTableFull);
  }
}

struct PartProbeParams {
  const PartEntry* entS;
  uint64_t n;
  uint32_t pbits;
  const unsigned long long* slot_off;
  const Slot* slots;
  VerifyParams V;      // arenas, offsets, ids, output (pairs, cap, count)
};

// S entries in partition order: each lane walks its entry's bucket sequence in
// its partition's table; candidates (signature and length equal) are compared
// byte for byte by the whole warp; verified pairs are staged per warp.
__global__ void __launch_bounds__(kVThreads, 4) part_probe_kernel(PartProbeParams Q) {
  __shared__ Stage stage_all[kVWarps];
  __shared__ uint4 emask[17];
  fill_emask(emask);
  __syncthreads();
  const VerifyParams& P = Q.V;
  const int lane = threadIdx.x & 31;
  Stage& stage = stage_all[threadIdx.x >> 5];
  uint32_t np = 0;
  const uint64_t ngroups = (Q.n + 31) / 32;
  const uint64_t nwarps = (uint64_t)gridDim.x * kVWarps;
  for (uint64_t grp = (uint64_t)blockIdx.x * kVWarps + (threadIdx.x >> 5); grp < ngroups; grp += nwarps) {
    const uint64_t v = grp * 32 + (uint64_t)lane;
    bool live = v < Q.n;
    uint64_t sig = 0, start = 0, len = 0, b = 0, msk = 0, steps = 0;
    uint32_t l32 = 0, srow = 0;
    const Slot* tab = Q.slots;
    if (live) {
      const PartEntry e = Q.entS[v];
      sig = e.sig;
      l32 = (uint32_t)(e.key >> 32);
      srow = (uint32_t)e.key;
      start = __ldg(P.offS + srow);
      len = __ldg(P.offS + srow + 1) - start;
      const uint64_t h = sig_hash(sig, l32);
      const uint32_t p = part_of(h, Q.pbits);
      tab = Q.slots + Q.slot_off[p];
      msk = Q.slot_off[p + 1] - Q.slot_off[p] - 1;
      b = h & msk;
    }
    while (__any_sync(kFull, live)) {
      bool cand = false;
      uint32_t row = 0;
      if (live) {
        const ulonglong2 s = __ldg(reinterpret_cast<const ulonglong2*>(tab + b));
        if (s.y == kEmpty) {
          live = false;
        } else {
          if (s.x == sig && (uint32_t)(s.y >> 32) == l32) {
            cand = true;
            row = (uint32_t)s.y;
          }
          b = (b + 1) & msk;
          if (++steps > msk) live = false;
        }
      }
      uint32_t cm = __ballot_sync(kFull, cand);
      while (cm) {
        const int j = __ffs(cm) - 1;
        cm &= cm - 1;
        const uint32_t rj = __shfl_sync(kFull, row, j);
        const uint32_t lj = __shfl_sync(kFull, l32, j);
        const uint64_t stj = __shfl_sync(kFull, start, j);
        const uint64_t rs = __ldg(P.offR + rj);
        bool eq;
        if (lj < kNarrowLen) {
          eq = warp_equal(P.arenaR + rs, P.arenaS + stj, lj, emask);
        } else {
          const uint64_t ls = __shfl_sync(kFull, len, j);
          eq = __ldg(P.offR + rj + 1) - rs == ls && warp_equal_wide(P.arenaR, rs, P.arenaS, stj, ls);
        }
        if (eq) {
          const uint32_t sj = __shfl_sync(kFull, srow, j);
          if (lane == 0) {
            stage.r[np] = rj;
            stage.s[np] = sj;
          }
          __syncwarp();
          if (++np == (uint32_t)kVStage) {
            flush_stage(stage, np, P);
            np = 0;
          }
        }
      }
    }
  }
  if (np) flush_stage(stage, np, P);
}

}  // namespace algsig
