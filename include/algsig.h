/*
 * algsig.h -- C ABI of the GB300 algebraic-signature equi-join library
 * (libalgsig.so).
 *
 * The method (Mokadem, Hameurlain, Morvan, "Equi join query acceleration
 * using algebraic signatures", IADIS 2008):
 *   - Section 3.1: a key P is a string of l symbols p_0 .. p_{l-1} of GF(2^16);
 *     its n-symbol algebraic signature is the vector
 *         sig^k(P) = sum_{i=0}^{l-1} p_i * alpha_k^i,   k = 1..n,
 *     with sums as XOR and products in GF(2^16).
 *   - Section 3.2, Figure 2: compute Sign(r) for every r in R, build a hash
 *     table H_sign of R's signatures, probe it with every s in S, output the
 *     matching tuples, materialise T.
 *   - Section 2: simple hash join (build on the smaller relation R, probe with
 *     the larger S).
 *
 * Fixed choices of this library (the paper leaves them open):
 *   f = 16, n = 4, alpha_k = x^k, field polynomial x^16 + x^12 + x^3 + x + 1;
 *   symbol p_i = byte[2i] | byte[2i+1] << 8, a missing high byte of an
 *   odd-length key is 0; the signature is packed in one uint64 with sig^k in
 *   bits [16(k-1), 16k).  Every candidate pair found through the signatures is
 *   verified byte for byte, so the join result is exactly the equi-join
 *       T = { (r.id, s.id) : len(r) == len(s) and bytes(r) == bytes(s) }.
 *
 * Data layout (all pointers named d_* are device pointers):
 *   relation  = packed byte arena + offsets + ids.  Key i is the byte range
 *               arena[off[i] .. off[i+1]); offsets are non-decreasing uint64.
 *               Keys are packed back to back with no alignment requirement.
 *               The arena's allocation must be readable up to the next 16-byte
 *               boundary after its last key byte (16-byte aligned chunks that
 *               hold a key byte are read whole), and the arena pointer must be
 *               16-byte aligned.  ids may be NULL: row i then has id i.
 *   signature = uint64 per key, layout above.
 *   pairs     = uint32[2*cnt] holding (r_id, s_id) pairs; order unspecified.
 *
 * Ownership and memory: the caller owns every buffer.  The library never
 * allocates device memory; it only keeps fixed-size tables in module-scope
 * device memory that is set up once per device on first use.  Workspace sizes
 * are queried with the *_bytes functions.
 *
 * Streams: every call is asynchronous on the given stream (a cudaStream_t
 * passed as void*, NULL = legacy default stream) unless it is given a host
 * pointer to return a count, in which case it synchronises that stream.
 *
 * Errors: every call returns an as_status; AS_OK is 0.  as_last_error()
 * gives a human-readable message for the calling thread's last failure.  No
 * C++ exception crosses this boundary.
 */
#ifndef ALGSIG_H_
#define ALGSIG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int as_status;
typedef void* as_stream;   /* cudaStream_t */

enum {
    AS_OK = 0,
    AS_ERR_INVALID = 1,      /* bad argument: null pointer, misaligned arena, size out of range */
    AS_ERR_NOMEM = 2,        /* workspace smaller than the queried size */
    AS_ERR_CAPACITY = 3,     /* more result pairs than cap_pairs; the exact count is still returned */
    AS_ERR_TABLE_FULL = 4,   /* a build could not place a row (cannot happen for load_factor <= 1) */
    AS_ERR_CUDA = 5,         /* a CUDA runtime error; the message holds cudaGetErrorString */
    AS_ERR_UNSUPPORTED = 6   /* no usable GPU (this library has no CPU fallback) */
};

/* Human-readable message for the calling thread's last non-OK status. */
const char* as_last_error(void);

/* Name of a status code. */
const char* as_status_string(as_status st);

/* Library version, as 10000*major + 100*minor + patch. */
int as_version(void);

/*
 * as_sig_compute -- algebraic signatures of n keys (Section 3.1).
 *   d_arena, d_off : the relation (see layout above), device memory
 *   n              : number of keys; d_off has n+1 entries
 *   d_sig_out      : uint64[n], device memory, written completely
 * Errors: AS_ERR_INVALID for null pointers with n > 0 or a misaligned arena;
 * AS_ERR_CUDA if the launch fails.
 */
as_status as_sig_compute(const uint8_t* d_arena, const uint64_t* d_off, uint64_t n,
                         uint64_t* d_sig_out, as_stream stream);

/*
 * Hash table of R's signatures (H_sign of Figure 2).  Open addressing with
 * linear probing over cap = next power of two >= m / load_factor slots; a slot
 * is one uint64 (32-bit fingerprint of the signature hash << 32 | R row), all
 * ones when empty.  R's signatures and key offsets are referenced by row.
 * The struct is plain data and is filled by as_join_build; the caller keeps
 * it (host memory) and passes it to as_join_probe.  The device buffers it
 * points to belong to the caller: the workspace given to as_join_build and
 * R's arena / offsets / ids, which must stay alive and unchanged while the
 * table is used.
 */
typedef struct as_table {
    uint64_t* slots;          /* device: cap slots */
    const uint64_t* sigR;     /* device: m signatures of R */
    const uint8_t* arenaR;    /* device */
    const uint64_t* offR;     /* device: m+1 */
    const uint32_t* idR;      /* device or NULL */
    uint32_t* flags;          /* device: error flags written by the build */
    uint64_t m;
    uint64_t cap;             /* power of two */
    uint32_t log2cap;
    uint32_t reserved;
} as_table;

/*
 * Workspace of as_join_build: the slots, R's signatures and the flags, each
 * 256-byte aligned.  load_factor must be in (0, 1].  Returns 0 for invalid
 * arguments.
 */
size_t as_join_table_bytes(uint64_t m, float load_factor);

/*
 * as_join_build -- build H_sign on R (Figure 2, "Build(R, H_sign)").
 *   d_ws, ws_bytes : device workspace of at least as_join_table_bytes(m, lf)
 *   d_arenaR, d_offR, d_idR, m : relation R (m < 2^32 - 1)
 *   d_sigR         : R's signatures if already computed (uint64[m], device),
 *                    or NULL: they are computed into the workspace
 *   load_factor    : table fill target in (0, 1]
 *   out            : host struct filled with the table description
 * Errors: AS_ERR_INVALID, AS_ERR_NOMEM (workspace too small), AS_ERR_CUDA.
 */
as_status as_join_build(void* d_ws, size_t ws_bytes, const uint8_t* d_arenaR, const uint64_t* d_offR,
                        const uint32_t* d_idR, uint64_t m, const uint64_t* d_sigR, float load_factor,
                        as_table* out, as_stream stream);

/*
 * as_join_probe -- probe H_sign with every key of S and emit the verified
 * matches (Figure 2, "Probe(H_sign, S); output the matching tuples").
 * S's signatures are computed on the fly; a candidate is a slot whose
 * fingerprint, full signature and key length all match, and it is emitted
 * only if its bytes equal the S key's bytes.
 *   t              : table from as_join_build (host struct)
 *   d_arenaS, d_offS, d_idS, n : relation S
 *   d_sigS_out     : uint64[n] device buffer to receive S's signatures, or NULL
 *   d_pairs        : uint32[2*cap_pairs] device buffer for (r_id, s_id) pairs
 *   cap_pairs      : capacity of d_pairs in pairs; pairs beyond it are counted
 *                    but not written
 *   d_count        : device uint64 receiving the total pair count
 *   h_count        : host uint64 or NULL.  If given, the stream is synchronised,
 *                    the count is copied here and the build's error flags are
 *                    checked: AS_ERR_CAPACITY if count > cap_pairs,
 *                    AS_ERR_TABLE_FULL if the build overflowed.
 * Errors: AS_ERR_INVALID, AS_ERR_CAPACITY, AS_ERR_TABLE_FULL, AS_ERR_CUDA.
 */
as_status as_join_probe(const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS,
                        const uint32_t* d_idS, uint64_t n, uint64_t* d_sigS_out, uint32_t* d_pairs,
                        uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count, as_stream stream);

/* Workspace of as_join: the table workspace plus the pair counter. */
size_t as_join_ws_bytes(uint64_t m, float load_factor);

/*
 * as_join -- the whole signature hash join T = Join(R, S) in one call:
 * signatures of R, build, probe with S (signatures, verification, compaction).
 * Arguments as for as_join_build and as_join_probe; d_ws must hold
 * as_join_ws_bytes(m, load_factor) bytes.  d_count may be NULL (the counter
 * then lives in the workspace).
 */
as_status as_join(const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR, uint64_t m,
                  const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint64_t n,
                  float load_factor, void* d_ws, size_t ws_bytes, uint32_t* d_pairs, uint64_t cap_pairs,
                  uint64_t* d_count, uint64_t* h_count, as_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* ALGSIG_H_ */
