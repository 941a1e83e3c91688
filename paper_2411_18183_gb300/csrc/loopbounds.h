// loopbounds.h -- loop bounds of the warp-wide byte comparison (the exact
// verification of every candidate pair that makes the join exact), shared by
// the device code and a host-compiled check of the bounds.
//
// The comparison of two len-byte keys runs in 32-bit offsets from the aligned
// 16-byte chunk that holds the S key's first byte (that byte at offset
// sa < 16); the R key's bytes sit d < 16 bytes further.  One step compares
// 1024 bytes, and every offset a step forms stays below
//     steps * 1024 + d + 16  <=  sa + len + 1023 + 15 + 16,
// which is below 2^32 for every len < kNarrowLen.  Longer keys are compared
// in 64-bit offsets.  The loop is counted in steps, so it ends by
// construction.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define ALGSIG_HD __host__ __device__ __forceinline__
#else
#define ALGSIG_HD inline
#endif

namespace algsig {

constexpr uint32_t kNarrowLen = 0xFFFFF000u;   // keys of 2^32 - 4096 bytes and more: 64-bit offsets

// 1024-byte steps of the 32-bit comparison of a key of len bytes (len < kNarrowLen)
// whose S copy starts at byte sa (< 16) of its aligned chunk
ALGSIG_HD uint32_t narrow_steps(uint32_t sa, uint32_t len) { return (uint32_t)(((uint64_t)sa + len + 1023u) >> 10); }

// the largest offset a step of that comparison forms, plus one (as a 64-bit
// value, so that a check can see whether it fits 32 bits); d < 16 is the R
// key's misalignment
ALGSIG_HD uint64_t narrow_offset_end(uint32_t sa, uint32_t len, uint32_t d) {
  return (uint64_t)narrow_steps(sa, len) * 1024u + d + 16u;
}

}  // namespace algsig
