// xs3_net.h -- written by gen_xs3.py; do not edit by hand.
//
// Bit-sliced Horner step of signature component 3 (sig^3 = sum_i p_i x^(3i),
// Section 3.1) over theta = x^1536, in the basis of GF(2^16) given in
// gen_xs3.py, and the map of its state to polynomial coordinates of D_b(x^6).
// 13 three-input XORs per 16-byte chunk.
#pragma once

namespace algsig {

// S <- S theta^4 + v3 theta^3 + v2 theta^2 + v1 theta + v0 (v3 last in the key)
__device__ __forceinline__ void xs3_chunk(uint32_t (&c)[16], uint32_t v0, uint32_t v1, uint32_t v2,
                                          uint32_t v3) {
  const uint32_t n0 = c[13] ^ c[14] ^ v0;
  const uint32_t n1 = c[5] ^ c[6] ^ v1;
  const uint32_t n2 = c[0] ^ c[4] ^ c[8];
  const uint32_t n3 = c[4] ^ c[8] ^ v3;
  const uint32_t n4 = c[13] ^ v2;
  const uint32_t n5 = c[1] ^ c[12] ^ c[14];
  const uint32_t n6 = c[4];
  const uint32_t n7 = c[6] ^ c[7] ^ c[8];
  const uint32_t n8 = c[2] ^ c[6] ^ c[14];
  const uint32_t n9 = c[5];
  const uint32_t n10 = c[3] ^ c[8];
  const uint32_t n11 = c[10];
  const uint32_t n12 = c[2] ^ c[9] ^ c[12];
  const uint32_t n13 = c[4] ^ c[7] ^ c[8] ^ c[9] ^ c[14];
  const uint32_t n14 = c[15];
  const uint32_t n15 = c[7] ^ c[11] ^ c[13];
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3; c[4] = n4; c[5] = n5; c[6] = n6; c[7] = n7;
  c[8] = n8; c[9] = n9; c[10] = n10; c[11] = n11; c[12] = n12; c[13] = n13; c[14] = n14; c[15] = n15;
}

// p_i: bit b = coefficient of x^i in D_b(x^6)
__device__ __forceinline__ void xs3_to_poly(const uint32_t (&c)[16], uint32_t (&p)[16]) {
  p[0] = c[0] ^ c[2] ^ c[10] ^ c[11] ^ c[12] ^ c[14];
  p[1] = c[2] ^ c[5] ^ c[7] ^ c[8] ^ c[9] ^ c[10] ^ c[11] ^ c[12] ^ c[15];
  p[2] = c[3] ^ c[7] ^ c[9] ^ c[12] ^ c[13] ^ c[15];
  p[3] = c[2] ^ c[3] ^ c[5] ^ c[7] ^ c[8] ^ c[11] ^ c[12] ^ c[13] ^ c[14];
  p[4] = c[2] ^ c[5] ^ c[8] ^ c[10] ^ c[11] ^ c[13] ^ c[14] ^ c[15];
  p[5] = c[2] ^ c[3] ^ c[5] ^ c[8] ^ c[9] ^ c[10] ^ c[13] ^ c[15];
  p[6] = c[1] ^ c[5] ^ c[8] ^ c[10] ^ c[12] ^ c[13] ^ c[14];
  p[7] = c[2] ^ c[5] ^ c[6] ^ c[7] ^ c[8] ^ c[9] ^ c[10] ^ c[11] ^ c[12] ^ c[13] ^ c[14];
  p[8] = c[2] ^ c[6] ^ c[7] ^ c[9] ^ c[10] ^ c[13] ^ c[14] ^ c[15];
  p[9] = c[2] ^ c[5] ^ c[7] ^ c[8] ^ c[10] ^ c[12] ^ c[15];
  p[10] = c[5] ^ c[7] ^ c[8] ^ c[9] ^ c[13] ^ c[15];
  p[11] = c[2] ^ c[5] ^ c[6] ^ c[7] ^ c[9] ^ c[10] ^ c[12] ^ c[13] ^ c[14];
  p[12] = c[2] ^ c[4] ^ c[7] ^ c[13] ^ c[14];
  p[13] = c[7] ^ c[9] ^ c[10] ^ c[11] ^ c[13];
  p[14] = c[3] ^ c[6] ^ c[7] ^ c[10] ^ c[11] ^ c[12] ^ c[14];
  p[15] = c[5] ^ c[6] ^ c[7] ^ c[8] ^ c[12] ^ c[14] ^ c[15];
}

}  // namespace algsig
