// gen_dev.cu -- the input generator on the device: the same relations as the
// host generator (gen.c) for joins without duplicated R keys, Zipf partners or
// near-duplicates (the batch and serving workloads), written straight into
// device memory, so that relations of hundreds of GB need no host copy.
//
// Holds no part of the join or signature arithmetic: only key bytes, lengths
// and the row plan, from the counter-based choices of genrng.h that the host
// generator uses too.  A "wave" is a run of joins packed back to back into one
// R and one S relation, as workloads.generate_batch packs them.
//
//   gd_plan : per row, its key's identity (relation bit 63 | identity) and
//             length (written to off[row + 1]; off[0] = 0)
//   (the caller turns the lengths into offsets with a prefix sum)
//   gd_fill : the key bytes of every row, and zeros up to the padded arena end
#include <cuda_runtime.h>
#include <stdint.h>

#define GEN_HD __host__ __device__
#include "genrng.h"

extern "C" {

// One join of a wave (host memory; gd_plan and gd_fill copy the table).
typedef struct {
    uint64_t seed;
    uint64_t m, n;                  // |R|, |S|
    uint64_t n_copy;                // S rows that copy an R key (llround(frac_copy * n))
    uint64_t r_row0, s_row0;        // first row of the join in the wave's R and S
    uint32_t r_len_lo, r_len_hi;    // R key length, uniform inclusive
    uint32_t s_len_lo, s_len_hi;    // fresh S key length, uniform inclusive
    int32_t alphabet;               // as in gen.c (4: XML-like text)
    int32_t reserved;
} gd_join;

}

namespace {

constexpr int kMaxJoins = 512;                 // the join table lives in constant memory (72 B a join)
__constant__ gd_join c_joins[kMaxJoins];

// join of a row: the last join whose first row is <= row
template <bool S_SIDE>
__device__ __forceinline__ int join_of_row(int nj, uint64_t row) {
    int lo = 0, hi = nj - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const uint64_t first = S_SIDE ? c_joins[mid].s_row0 : c_joins[mid].r_row0;
        if (first <= row) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr uint64_t kRelBit = 1ull << 63;

// row plan: identity and length of every row's key (R rows, then S rows)
__global__ void plan_kernel(int nj, uint64_t mR, uint64_t nS, uint64_t* offR, uint64_t* identR, uint64_t* offS,
                            uint64_t* identS) {
    const uint64_t total = mR + nS;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        if (i < mR) {
            const gd_join& J = c_joins[join_of_row<false>(nj, i)];
            const uint64_t r = i - J.r_row0;
            const uint64_t ident = gen_perm(J.seed, T_PERM_R, J.m, r);   // R keys are all distinct
            identR[i] = ident;
            offR[i + 1] = gen_key_len(J.seed, 0, ident, J.r_len_lo, J.r_len_hi);
        } else {
            const uint64_t row = i - mR;
            const gd_join& J = c_joins[join_of_row<true>(nj, row)];
            const uint64_t j = row - J.s_row0;
            const uint64_t p = gen_perm(J.seed, T_PERM_S, J.n, j);
            if (J.m > 0 && p < J.n_copy) {                             // a copy of R row u % m's key
                const uint64_t r = gen_rnd(J.seed, T_PARTNER, j, 0) % J.m;
                const uint64_t ident = gen_perm(J.seed, T_PERM_R, J.m, r);
                identS[row] = ident;
                offS[row + 1] = gen_key_len(J.seed, 0, ident, J.r_len_lo, J.r_len_hi);
            } else {                                                   // a fresh key
                identS[row] = kRelBit | j;
                offS[row + 1] = gen_key_len(J.seed, 1, j, J.s_len_lo, J.s_len_hi);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        offR[0] = 0;
        offS[0] = 0;
    }
}

// key bytes: one warp per row (letters, 4 bytes per random word), or one
// thread per row for XML-like text (its elements are drawn in sequence)
template <bool S_SIDE>
__global__ void fill_kernel(int nj, uint64_t rows, const uint64_t* off, const uint64_t* ident, uint8_t* arena,
                            int xml) {
    if (xml) {
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
             i += (uint64_t)gridDim.x * blockDim.x) {
            const gd_join& J = c_joins[join_of_row<S_SIDE>(nj, i)];
            const uint64_t id = ident[i];
            gen_xml_bytes(J.seed, T_BYTE + 16 * (id >> 63), id & ~kRelBit, arena + off[i], off[i + 1] - off[i]);
        }
        return;
    }
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < rows; i += nwarps) {
        const gd_join& J = c_joins[join_of_row<S_SIDE>(nj, i)];
        const uint64_t id = ident[i];
        const uint64_t rel = id >> 63, idn = id & ~kRelBit;
        const uint64_t b = off[i], len = off[i + 1] - b;
        for (uint64_t g = lane; 4 * g < len; g += 32) {
            const uint64_t r = gen_group_word(J.seed, rel, idn, g);
            for (int q = 0; q < 4 && 4 * g + q < len; q++)
                arena[b + 4 * g + q] = gen_letter(J.alphabet, (uint16_t)(r >> (16 * q)));
        }
    }
}

int blocks_for(uint64_t work, int per_block) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (work + per_block - 1) / per_block;
    const uint64_t lim = (uint64_t)(sms > 0 ? sms : 1) * 32;
    return (int)(want < 1 ? 1 : (want < lim ? want : lim));
}

}  // namespace

extern "C" {

// Largest join count of one call.
int gd_max_joins(void) { return kMaxJoins; }

// Row plan of a wave: offR (uint64[mR + 1]) and offS (uint64[nS + 1]) get
// 0 at index 0 and the key length of row i at index i + 1; identR / identS
// (uint64[mR] / uint64[nS]) the key identities.  All device memory.  The
// joins must be in row order, their alphabets equal.  Returns 0, or a
// cudaError_t.  The join table is held in one constant buffer: calls on
// different streams must not overlap.
int gd_plan(const gd_join* joins, int nj, uint64_t mR, uint64_t nS, uint64_t* offR, uint64_t* identR, uint64_t* offS,
            uint64_t* identS, cudaStream_t stream) {
    if (nj < 1 || nj > kMaxJoins) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyToSymbolAsync(c_joins, joins, sizeof(gd_join) * nj, 0, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return (int)e;
    plan_kernel<<<blocks_for(mR + nS, 256), 256, 0, stream>>>(nj, mR, nS, offR, identR, offS, identS);
    return (int)cudaGetLastError();
}

// Key bytes of one side of a wave (side 0: R, 1: S) from its offsets (after
// the prefix sum) and identities; the arena (device) must hold off[rows]
// bytes, and bytes [off[rows], arena_bytes) are set to zero.  off and ident
// index the rows of `joins`, whose r_row0 / s_row0 count from the first of them.
int gd_fill(const gd_join* joins, int nj, int side, uint64_t rows, const uint64_t* off, const uint64_t* ident,
            uint8_t* arena, uint64_t arena_bytes, uint64_t key_bytes, cudaStream_t stream) {
    if (nj < 1 || nj > kMaxJoins || key_bytes > arena_bytes) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyToSymbolAsync(c_joins, joins, sizeof(gd_join) * nj, 0, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return (int)e;
    if (arena_bytes > key_bytes && (e = cudaMemsetAsync(arena + key_bytes, 0, arena_bytes - key_bytes, stream)) != cudaSuccess)
        return (int)e;
    if (rows == 0) return 0;
    const int xml = joins[0].alphabet == 4;
    const int blocks = xml ? blocks_for(rows, 128) : blocks_for(rows * 32, 256);
    if (side) fill_kernel<true><<<blocks, xml ? 128 : 256, 0, stream>>>(nj, rows, off, ident, arena, xml);
    else fill_kernel<false><<<blocks, xml ? 128 : 256, 0, stream>>>(nj, rows, off, ident, arena, xml);
    return (int)cudaGetLastError();
}

}
