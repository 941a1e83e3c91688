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
 * are queried with the *_bytes functions.  cudaDeviceReset discards those
 * tables (and as_join_probe_noalloc's scratch address) without the library
 * noticing: do not call the library on a device again after resetting it in
 * the same process.
 *
 * Streams: every call is asynchronous on the given stream (a cudaStream_t
 * passed as void*, NULL = legacy default stream) unless it is given a host
 * pointer to return a count, in which case it synchronises that stream.
 * as_join (below 2^19 S keys), as_join_batch_run and as_baseline_join run
 * S's signatures (or hashes) on a side stream of the library (four per
 * device, created with the tables) forked from the given stream and joined
 * back into it before the probe, so that they overlap R's signatures and the
 * build; the calls stay asynchronous on the given stream and can be captured
 * in a CUDA graph.
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
 * as_sig_compute_n -- as_sig_compute with n_components = n of Section 3.1:
 * 4 (the same result as as_sig_compute) or 2 (the paper's two-symbol
 * signature sig_{alpha,2} of Sections 3.1 and 4.3, 4 bytes: components 1 and 2
 * in bits 0..31, bits 32..63 zero).  A join on two-component signatures is
 * as_join_build with d_sigR and as_join_probe_mode with d_sigS, both from
 * this call with n_components = 2; the table and probe compare the 64-bit
 * words, so only the two components take part.
 * Errors: as for as_sig_compute, and AS_ERR_INVALID for n_components other
 * than 2 or 4.
 */
as_status as_sig_compute_n(const uint8_t* d_arena, const uint64_t* d_off, uint64_t n, int n_components,
                           uint64_t* d_sig_out, as_stream stream);

/*
 * Launch shapes of the signature kernel of as_sig_compute (Section 3.1 fixes
 * the result, not the schedule): shape s runs warps[s] warps per block, one
 * key per lane, with depth[s] 32-byte blocks of each key in flight.  Every
 * shape gives the same signatures; which is fastest depends on the key-length
 * mix, so a tuner times them.  Shape 0 is the default of as_sig_compute.
 *
 * as_sig_shapes -- writes up to cap (warps, depth) pairs (either array may be
 *   null) and returns the number of shapes.
 * as_sig_compute_shape -- as_sig_compute_n with an explicit shape.  Errors: as
 *   for as_sig_compute_n, and AS_ERR_INVALID for a shape outside
 *   [0, as_sig_shapes(0, 0, 0)).
 */
int as_sig_shapes(int* warps, int* depth, int cap);
as_status as_sig_compute_shape(const uint8_t* d_arena, const uint64_t* d_off, uint64_t n, int n_components,
                               int shape, uint64_t* d_sig_out, as_stream stream);

/*
 * as_sig_compute_gf8 -- signatures with byte symbols (Section 3.1: a symbol
 * is a byte or a double byte): GF(2^8) with field polynomial
 * x^8 + x^4 + x^3 + x^2 + 1, alpha_k = x^k, p_i = byte i,
 *     sig8^k = sum_{i=0}^{l-1} b_i x^(k i),   k = 1..4,
 * packed with component k in bits [8(k-1), 8k) (bits 32..63 zero).  Keys of
 * equal length under 255 bytes that differ in at most 4 bytes have different
 * signatures; past 255 bytes the exponent wraps (x^255 = 1).  A join on them is
 * as_join_build with d_sigR and as_join_probe_mode with d_sigS, both from this
 * call.  Arguments and errors as for as_sig_compute.
 */
as_status as_sig_compute_gf8(const uint8_t* d_arena, const uint64_t* d_off, uint64_t n, uint64_t* d_sig_out,
                             as_stream stream);

/*
 * Cumulative (prefix) signatures (Section 5 lists them, after the paper's
 * reference [7], as the way to signatures of prefixes and substrings).  For a
 * block size B (a positive multiple of 16 bytes) key i of length len gets
 * max(1, ceil(len / B)) entries
 *     C_j = sig(key[0 .. min((j+1) B, len))),   j = 0, 1, ...
 * (a single 0 for the empty key); its last entry is sig(key).  By the
 * concatenation rule of Section 3.1, the signature of any substring starting
 * at an even byte a < b is x^(-k a/2) (C(b) + C(a)) component-wise, with C(a)
 * the signature of the a-byte prefix (a block boundary when a is a multiple
 * of B).
 *
 * as_sig_prefix_offsets -- layout of the entries: d_pref_off[i] (uint64[n+1],
 *   device) receives the index of key i's first entry, d_pref_off[n] the total
 *   count.  d_ws: device workspace of as_sig_prefix_ws_bytes(n) bytes.
 *   Errors: AS_ERR_INVALID (block size, null pointers), AS_ERR_NOMEM, AS_ERR_CUDA.
 * as_sig_prefixes -- the entries: d_out (uint64[d_pref_off[n]], device)
 *   receives key i's entries at d_out[d_pref_off[i] ...], packed like
 *   as_sig_compute.  d_pref_off as written by as_sig_prefix_offsets with the
 *   same block size.  Errors: as for as_sig_compute, and AS_ERR_INVALID for a
 *   block size that is not a positive multiple of 16.
 */
size_t as_sig_prefix_ws_bytes(uint64_t n);
as_status as_sig_prefix_offsets(const uint64_t* d_off, uint64_t n, uint32_t block_bytes, uint64_t* d_pref_off,
                                void* d_ws, size_t ws_bytes, as_stream stream);
as_status as_sig_prefixes(const uint8_t* d_arena, const uint64_t* d_off, uint64_t n, uint32_t block_bytes,
                          const uint64_t* d_pref_off, uint64_t* d_out, as_stream stream);

/*
 * Hash table of R's signatures (H_sign of Figure 2).  Open addressing with
 * linear probing over cap = next power of two >= max(64, m / load_factor)
 * slots of 16 bytes: the R row's 64-bit signature, then one uint64 holding
 * (min(key length, 2^32 - 2) << 32) | R row, all ones when the slot is empty.
 * The bucket of a key is a hash of its signature and length.
 * The struct is plain data and is filled by as_join_build; the caller keeps
 * it (host memory) and passes it to as_join_probe.  The device buffers it
 * points to belong to the caller: the workspace given to as_join_build and
 * R's arena / offsets / ids, which must stay alive and unchanged while the
 * table is used.
 */
typedef struct as_table {
    uint64_t* slots;          /* device: cap slots of two uint64 */
    const uint64_t* sigR;     /* device: m signatures of R */
    const uint8_t* arenaR;    /* device */
    const uint64_t* offR;     /* device: m+1 */
    const uint32_t* idR;      /* device or NULL */
    uint32_t* flags;          /* device: error flags written by the build */
    uint64_t m;
    uint64_t cap;             /* power of two */
    uint32_t log2cap;
    uint32_t reserved;
    uint32_t* matched;        /* device: ceil(m/32) words, one bit per R row, set by
                                 the R-side output modes of as_join_probe_mode;
                                 NULL: the table supports no R-side mode */
} as_table;

/*
 * Workspace of as_join_build: the slots (16 bytes each), R's signatures, the
 * flags and a bitmap of R's rows (for the R-side output modes of
 * as_join_probe_mode), each 256-byte aligned.  load_factor must be in (0, 1].
 * Returns 0 for invalid arguments.
 */
size_t as_join_table_bytes(uint64_t m, float load_factor);

/*
 * as_join_build -- build H_sign on R (Figure 2, "Build(R, H_sign)").
 *   d_ws, ws_bytes : device workspace of at least as_join_table_bytes(m, lf)
 *   d_arenaR, d_offR, d_idR, m : relation R (m < 2^32 - 1)
 *   d_sigR         : R's signatures if already computed (uint64[m], device),
 *                    or NULL: they are computed into the workspace by the
 *                    kernel that inserts them (signatures and build in one
 *                    pass over R's keys)
 *   load_factor    : table fill target in (0, 1]
 *   out            : host struct filled with the table description
 * Errors: AS_ERR_INVALID, AS_ERR_NOMEM (workspace too small), AS_ERR_CUDA.
 */
as_status as_join_build(void* d_ws, size_t ws_bytes, const uint8_t* d_arenaR, const uint64_t* d_offR,
                        const uint32_t* d_idR, uint64_t m, const uint64_t* d_sigR, float load_factor,
                        as_table* out, as_stream stream);

/* Workspace of as_join_probe when it must keep S's signatures itself
 * (d_sigS_out == NULL): n signatures, 256-byte aligned. */
size_t as_join_probe_ws_bytes(uint64_t n);

/*
 * as_join_probe -- probe H_sign with every key of S and emit the verified
 * matches (Figure 2, "Probe(H_sign, S); output the matching tuples").
 * S's signatures are computed first (as by as_sig_compute); then every S key
 * walks its bucket sequence until an empty slot; a slot is a candidate when
 * its signature and key length equal the S key's, and a candidate is emitted
 * only if the R key's bytes equal the S key's bytes.  From 2^19 S keys the
 * two steps run as one kernel (each group of 32 keys is probed and verified
 * right after its signatures), with the same result.
 *   t              : table from as_join_build (host struct)
 *   d_arenaS, d_offS, d_idS, n : relation S
 *   d_sigS_out     : uint64[n] device buffer to receive S's signatures, or NULL
 *   d_ws, ws_bytes : device workspace of as_join_probe_ws_bytes(n) bytes,
 *                    256-byte aligned; used (and required) only when
 *                    d_sigS_out is NULL
 *   d_pairs        : uint32[2*cap_pairs] device buffer for (r_id, s_id) pairs,
 *                    8-byte aligned
 *   cap_pairs      : capacity of d_pairs in pairs; pairs beyond it are counted
 *                    but not written
 *   d_count        : device uint64 receiving the total pair count
 *   h_count        : host uint64 or NULL.  If given, the stream is synchronised,
 *                    the count is copied here and the build's error flags are
 *                    checked: AS_ERR_CAPACITY if count > cap_pairs,
 *                    AS_ERR_TABLE_FULL if the build overflowed.
 * Errors: AS_ERR_INVALID, AS_ERR_NOMEM, AS_ERR_CAPACITY, AS_ERR_TABLE_FULL,
 * AS_ERR_CUDA.
 */
as_status as_join_probe(const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS,
                        const uint32_t* d_idS, uint64_t n, uint64_t* d_sigS_out, void* d_ws, size_t ws_bytes,
                        uint32_t* d_pairs, uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count,
                        as_stream stream);

/*
 * as_join_probe_sigs -- as_join_probe with S's signatures already computed
 * by as_sig_compute: the second half of the probe step of Section 4.1,
 * formula 4 (compute sig(S_i), then probe H_sign with it), for callers that
 * keep signatures with a relation or time the two halves apart.  Only the
 * table walk, verification and compaction run.
 *   d_sigS         : uint64[n] device buffer holding sig(S_i) for every row i
 *                    (read only; wrong signatures only lose matches, the
 *                    byte-exact verification still rejects non-matches)
 * Other arguments, results and errors as for as_join_probe.
 */
as_status as_join_probe_sigs(const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS,
                             const uint32_t* d_idS, uint64_t n, const uint64_t* d_sigS, uint32_t* d_pairs,
                             uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count, as_stream stream);

/*
 * Output modes of as_join_probe_mode (the left, right and semi-join variants
 * that Section 5 lists as extensions; R is the build side, S the probe side).
 *   AS_JOIN_INNER   : the (r_id, s_id) pairs, as as_join_probe
 *   AS_JOIN_SEMI    : one (AS_NO_ROW, s_id) per S row with at least one match
 *   AS_JOIN_ANTI    : one (AS_NO_ROW, s_id) per S row with no match
 *   AS_JOIN_OUTER_S : the inner pairs plus one (AS_NO_ROW, s_id) per S row
 *                     with no match (outer join preserving S)
 *   AS_JOIN_OUTER_R : the inner pairs plus one (r_id, AS_NO_ROW) per R row
 *                     with no match (outer join preserving R)
 *   AS_JOIN_SEMI_R  : one (r_id, AS_NO_ROW) per R row with at least one match
 *   AS_JOIN_ANTI_R  : one (r_id, AS_NO_ROW) per R row with no match
 *                     (the R-side modes mark R's matched rows in the table's
 *                     bitmap during the probe, then list the selected rows;
 *                     they need a table from as_join_build, and two R-side
 *                     probes of one table must not overlap)
 *   AS_JOIN_SIG_ONLY: the probe of Figure 2 as the paper runs it: one
 *                     (r_id, s_id) pair per slot whose signature and key
 *                     length equal the S key's, with no byte comparison.
 *                     NOT exact: two different keys of equal length and equal
 *                     signatures are paired (keys that differ in at most n
 *                     symbols, n the signature's components, never are:
 *                     Section 3.1); its count minus the INNER count is the
 *                     number of signature collisions among the candidates.
 */
enum {
    AS_JOIN_INNER = 0,
    AS_JOIN_SEMI = 1,
    AS_JOIN_ANTI = 2,
    AS_JOIN_OUTER_S = 3,
    AS_JOIN_SIG_ONLY = 4,
    AS_JOIN_OUTER_R = 5,
    AS_JOIN_SEMI_R = 6,
    AS_JOIN_ANTI_R = 7
};
#define AS_NO_ROW 0xFFFFFFFFu

/*
 * as_join_probe_mode -- as_join_probe_sigs (S's signatures given, from
 * as_sig_compute) with an output mode.  Matches are exact (byte-verified) in
 * every mode but AS_JOIN_SIG_ONLY.  d_pairs receives the mode's output records as (r_id, s_id)
 * pairs in unspecified order; d_count / h_count count them.  Errors as for
 * as_join_probe, and AS_ERR_INVALID for an unknown mode.
 */
as_status as_join_probe_mode(const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS,
                             const uint32_t* d_idS, uint64_t n, const uint64_t* d_sigS, int mode, uint32_t* d_pairs,
                             uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count, as_stream stream);

/* Workspace of as_join for |R| = m and |S| = n: the table workspace, the pair
 * counter and the probe workspace. */
size_t as_join_ws_bytes(uint64_t m, uint64_t n, float load_factor);

/*
 * as_join -- the whole signature hash join T = Join(R, S) in one call:
 * signatures of R, build, probe with S (signatures, verification, compaction).
 * Arguments as for as_join_build and as_join_probe; d_ws must hold
 * as_join_ws_bytes(m, load_factor) bytes.  d_count may be NULL (the counter
 * then lives in the workspace).  R's signatures and the build are one kernel.
 * From 2^19 S keys it is as_join_build then as_join_probe (whose signatures
 * and probe then run as one kernel too: one pass over each relation's keys);
 * below that, S's signatures overlap R's pass on a side stream.  The result is
 * the same either way.
 */
as_status as_join(const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR, uint64_t m,
                  const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint64_t n,
                  float load_factor, void* d_ws, size_t ws_bytes, uint32_t* d_pairs, uint64_t cap_pairs,
                  uint64_t* d_count, uint64_t* h_count, as_stream stream);

/*
 * Prefix join: the join on the keys' first L bytes,
 *     T_L = {(r.id, s.id) : r.key[0 .. min(L, |r|)) == s.key[0 .. min(L, |s|))},
 * byte strings equal (so of equal length).  The signature of a key's L-byte
 * prefix is its cumulative signature at L (Section 5's cumulative
 * signatures); the build, probe and verification run on the truncated keys.
 * With L at least the longest key it is as_join's result; with L = 0 every
 * pair joins.
 *
 * as_join_prefix_ws_bytes -- workspace (0 for a bad load factor or m >= 2^32-1).
 * as_join_prefix -- arguments as for as_join, plus prefix_len = L
 *   (0 <= L <= 2^32 - 16).  Errors as for as_join_partitioned.
 */
size_t as_join_prefix_ws_bytes(uint64_t m, uint64_t n, float load_factor);
as_status as_join_prefix(const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR, uint64_t m,
                         const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint64_t n,
                         uint64_t prefix_len, float load_factor, void* d_ws, size_t ws_bytes, uint32_t* d_pairs,
                         uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count, as_stream stream);

/*
 * Radix-partitioned join: the same result as as_join, with R and S first split
 * into 2^part_bits partitions by the top bits of the bucket hash of (signature,
 * length), each partition joined with its own table (the partitioned, Grace
 * style hash join of Sections 2 and 4, in device memory).  Partitions hold
 * (signature, length | row) entries, not key bytes; the probe walks S in
 * partition order and verifies candidates byte for byte from the arenas.
 *
 * as_join_part_ws_bytes -- workspace for |R| = m, |S| = n (0 for a load factor
 *   outside (0, 1], m >= 2^32 - 1, n >= 2^32 or part_bits > 12).
 * as_join_partitioned -- arguments as for as_join, plus part_bits: the number
 *   of partition bits, 0..12, or AS_PART_BITS_AUTO (about 1024 R rows per
 *   partition).  Errors: AS_ERR_INVALID (bad argument, misaligned arena or
 *   pair buffer), AS_ERR_NOMEM (workspace too small), AS_ERR_TABLE_FULL,
 *   AS_ERR_CAPACITY (more pairs than cap_pairs; the count is still written),
 *   AS_ERR_CUDA.  Synchronises the stream when h_count is not NULL.
 */
#define AS_PART_BITS_AUTO 0xFFFFFFFFu
size_t as_join_part_ws_bytes(uint64_t m, uint64_t n, float load_factor, uint32_t part_bits);
as_status as_join_partitioned(const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR, uint64_t m,
                              const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint64_t n,
                              float load_factor, uint32_t part_bits, void* d_ws, size_t ws_bytes, uint32_t* d_pairs,
                              uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count, as_stream stream);

/*
 * Batches of independent joins (many joins of uneven sizes and key lengths in
 * one set of launches).  All joins' R relations are packed into one R
 * relation (one arena, one offset array) and all S relations into one S
 * relation; join j owns R rows [r_begin, r_end) and S rows [s_begin, s_end)
 * (ranges in increasing order, not overlapping), its own hash table (sized by
 * its own |R|) and its own output region: pairs [pair_offset, pair_offset +
 * pair_cap) of d_pairs, with its pair count in d_counts[j].  Pair ids are
 * the relations' ids if given, else row numbers relative to the join's first
 * row.  Per join the result is exactly that of as_join on the join's rows.
 * Only the rows inside the joins' ranges are read, so a batch may pick any
 * ordered subset of joins out of a larger resident pool (mR / nS are the
 * pool relations' sizes).
 */
typedef struct as_join_desc {
    uint64_t r_begin, r_end;
    uint64_t s_begin, s_end;
    uint64_t pair_offset;
    uint64_t pair_cap;
} as_join_desc;

/* Prepared batch: device descriptors and workspace regions (plain data).
 * mR / nS here count the rows of the batch's joins only. */
typedef struct as_batch {
    void* descs;
    uint64_t* slots;
    uint64_t* sigR;
    uint64_t* sigS;
    uint32_t* flags;
    uint64_t n_joins;
    uint64_t slots_total;
    uint64_t mR, nS;
    /* First row of the batch's R (S) rows when the joins' row ranges, taken in
     * join order, form one ascending contiguous range (the signatures then run
     * as those of a single relation); AS_ROWS_SCATTERED otherwise. */
    uint64_t r_first, s_first;
    /* Shape of the signature kernel for a side whose rows form one run (see
     * as_sig_shapes); as_join_batch_prepare sets 0, a tuner may change it
     * before as_join_batch_run. */
    int32_t sig_shape;
    int32_t reserved0;
} as_batch;
#define AS_ROWS_SCATTERED (~(uint64_t)0)

/* Workspace of a batch (0 for invalid descriptors or load factor). */
size_t as_join_batch_ws_bytes(const as_join_desc* descs, int n_joins, uint64_t mR, uint64_t nS, float load_factor);

/* Lay out the workspace and upload the descriptors (host array, copied; the
 * stream is synchronised once).  The prepared batch can be run many times, and
 * as_join_batch_run can be captured in a CUDA graph. */
as_status as_join_batch_prepare(const as_join_desc* descs, int n_joins, uint64_t mR, uint64_t nS, float load_factor,
                                void* d_ws, size_t ws_bytes, as_batch* out, as_stream stream);

/* Run a prepared batch: clear the tables and counters, signatures of all R
 * keys, build of every join's table, signatures of all S keys, probe and
 * verification of every S key against its join's table.  The signatures of a
 * side whose rows form one run (r_first / s_first set) come from the
 * signature kernel of as_sig_compute over that run; scattered rows take the
 * same kernel over the joins' row ranges back to back (its windows of keys
 * end with each join's rows); both at the shape b->sig_shape.  Asynchronous;
 * a join's count may exceed its pair_cap (the excess pairs are not written). */
as_status as_join_batch_run(const as_batch* b, const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR,
                            const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint32_t* d_pairs,
                            uint64_t* d_counts, as_stream stream);

/* prepare + run */
as_status as_join_batch(const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR, uint64_t mR,
                        const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint64_t nS,
                        const as_join_desc* descs, int n_joins, float load_factor, void* d_ws, size_t ws_bytes,
                        uint32_t* d_pairs, uint64_t* d_counts, as_stream stream);

/*
 * Comparison join (not the paper's method): the simple hash join on full
 * strings that the paper measures against (Section 2; Section 4.3 compares
 * with a join that tests a.equal(b) on every bucket entry).  The bucket is a
 * 64-bit hash of all key bytes; a slot holds the R row (tagged = 0), or the
 * R row and a 32-bit tag of the key hash (tagged = 1, an honesty control that
 * filters like a signature would).  Every visited slot costs a length check
 * and, when the lengths agree (and the tag matches, if tagged), a full byte
 * comparison.  Same output and errors as as_join.
 */
size_t as_baseline_ws_bytes(uint64_t m, uint64_t n, float load_factor);
as_status as_baseline_join(const uint8_t* d_arenaR, const uint64_t* d_offR, const uint32_t* d_idR, uint64_t m,
                           const uint8_t* d_arenaS, const uint64_t* d_offS, const uint32_t* d_idS, uint64_t n,
                           float load_factor, int tagged, void* d_ws, size_t ws_bytes, uint32_t* d_pairs,
                           uint64_t cap_pairs, uint64_t* d_count, uint64_t* h_count, as_stream stream);

/*
 * as_join_probe_noalloc -- as_join_probe with no workspace and no allocation
 * of any kind.  The paper has no counterpart: it is an interface for callers
 * that cannot allocate device memory at call time, e.g. a host engine that has
 * handed all device memory to its own pool (a serving process whose admission
 * budget accounts for every byte) or a latency-sensitive caller that must not
 * reach cudaMalloc/cudaFree (cudaFree synchronises the whole device).
 *
 * S's signatures go to a fixed scratch array compiled into the library
 * (AS_PROBE_NOALLOC_MAX_KEYS uint64 entries, 8 MiB per device), so:
 *   n              : at most AS_PROBE_NOALLOC_MAX_KEYS; larger n is rejected
 *                    with AS_ERR_INVALID before any device work
 *   nothing has to start at zero: the scratch is written completely before
 *   it is read, and d_count is cleared by the call itself
 *   calls that overlap on one device (two streams, or two host threads)
 *   share the scratch and race: serialise them, e.g. on one stream
 * The first call on a device (with that device current) does one-time setup:
 * the library's tables and kernel attributes, and the scratch address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The address is kept for the life of the process (see cudaDeviceReset
 * above).  Error messages name as_join_probe_noalloc.
 * Other arguments, results and errors as for as_join_probe with
 * d_sigS_out = NULL.
 */
#define AS_PROBE_NOALLOC_MAX_KEYS (1u << 20)
as_status as_join_probe_noalloc(const as_table* t, const uint8_t* d_arenaS, const uint64_t* d_offS,
                                const uint32_t* d_idS, uint64_t n, uint32_t* d_pairs, uint64_t cap_pairs,
                                uint64_t* d_count, uint64_t* h_count, as_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* ALGSIG_H_ */
