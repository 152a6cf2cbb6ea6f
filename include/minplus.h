/*
 * minplus.h -- C ABI of the GB300 (sm_103a) library for exact integer
 * (min,+) matrix products and the 2-domination power chain of
 * arXiv 2409.17688 ("HPC acceleration of large (min,+) matrix products to
 * compute domination-type parameters in graphs").
 *
 * Notation.  The paper writes the cylinder as P_m x C_n with m the path
 * order.  This library writes P_n x C_m: n is the path order (it fixes the
 * matrix size N = |C_n|, Table 1) and m is the cycle length (the power).
 *
 * Conventions shared by every entry point.
 *  - Matrices are row-major with a leading dimension counted in elements.
 *  - "device" pointers are CUDA device memory owned by the caller (for
 *    example torch tensors); "host" pointers are ordinary host memory.
 *    The library never frees caller memory.  It owns only the internal
 *    scratch it allocates (stream-ordered, freed before the call's work
 *    completes on the stream) and the per-device caches listed below.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued asynchronously on it unless an entry point
 *    says it is synchronous.  Entry points that must size internal buffers
 *    from device data synchronize the stream once; each says so.
 *  - INF encoding: 0x7FFF for int16 (MP_I16) and 255 for uint8 (MP_U8).
 *    Every input entry must lie in [0, INF].  Products are saturating:
 *    result = min(INF, min_l X_il + Y_lj), so an INF entry never produces a
 *    finite value.  Outside [0, INF] the results are unspecified.
 *  - Every function returns MP_OK (0) or a negative status; the message of
 *    the last failure on the calling host thread is in mp_last_error().
 *  - Asynchronous device-side failures (a bounded wait that ran out) are
 *    latched in a per-device flag read by mp_device_status().
 */
#ifndef MINPLUS_H
#define MINPLUS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MP_OK 0
#define MP_EINVAL -1   /* bad argument: n, m, k_max, sizes, leading dims, dtype */
#define MP_EALIAS -2   /* an output buffer overlaps an input buffer            */
#define MP_ENOMEM -3   /* device or host allocation failed / does not fit HBM  */
#define MP_ERANGE -4   /* exact result could reach the INF code (m*n >= 32767) */
#define MP_ECUDA -5    /* a CUDA runtime call failed                           */
#define MP_ETIMEOUT -6 /* a bounded device-side wait ran out                   */
#define MP_EBUSY -7    /* a server queue is full                               */
#define MP_ENOTREADY -8 /* a polled server ticket has not finished yet          */
#define MP_EIO -9      /* a file cannot be read or written, or is not a checkpoint
                          of this library's powers                            */
#define MP_ECHECK -10  /* a bounds-checked build (compiled with -DMP_CHECK)
                          caught an index outside its buffer                  */

/* ---- element types ----------------------------------------------------- */
#define MP_I16 0 /* int16 entries in [0, 0x7FFF], INF = 0x7FFF */
#define MP_U8 1  /* uint8 entries in [0, 255],    INF = 255    */

#define MP_INF16 0x7FFF
#define MP_INF8 0xFF

/* Largest path order the library enumerates (words are packed 2 bits per
 * letter in 32 bits).  The dense A(D_n) fits one GB300 up to n = 13. */
#define MP_MAX_PATH_ORDER 16

/* ---- a1: correct words --------------------------------------------------
 * Section 2.2 (correct n-words) and Table 1 (their number).
 * mp_transfer_size returns N = |C_n|, the number of correct n-words, or a
 * negative status for n < 1 or n > MP_MAX_PATH_ORDER.  Host only, no CUDA.
 */
int64_t mp_transfer_size(int n);

/* The reuse circuit of A(D_n)'s sparse step on the current device (built
 * with the transfer plan on first use; no step runs).  A row of a product
 * A (x) X is the minimum, over its arcs q -> p, of z_p + X[p]; when the arcs
 * out of q' are a subset of those out of q, row q' of the result is part of
 * row q's minimum, so the step computes each row from a few result rows
 * (its cover) and the arcs they leave out, in levels.  Writes into the HOST
 * array info[0..cap): {columns per CTA chunk (0: the step runs without a
 * circuit), levels, row reads per column, of them result rows, nnz(A), N}.
 * Returns the number of fields written (at most 6), or a negative status. */
int mp_transfer_circuit_info(int n, int64_t *info, int cap);

/* Writes the correct n-words into the HOST array words[0..cap) in
 * lexicographic order (letter 1 most significant, 0 < 1 < 2), each packed
 * two bits per letter with letter 1 in bits 2(n-1)..2n-1, so the packed
 * values increase strictly.  Returns N (words beyond cap are not written),
 * or MP_EINVAL.  Host only. */
int64_t mp_transfer_words(int n, uint32_t *words, int64_t cap);

/* ---- a2: the transfer matrix A(D_n) -------------------------------------
 * Algorithm 1 with the arc rule and labels of Section 2.2: A[q][p] = number
 * of zeros of p when word p can follow word q, else INF16.  Row q is the
 * source column word, column p the target (Theorem 2).
 * A: DEVICE int16, N x N, leading dimension lda >= N (N from
 * mp_transfer_size).  words_opt: DEVICE uint32[N] receiving the packed
 * words, or NULL.  Asynchronous on stream (the word list is uploaded from a
 * pageable host buffer).  Errors: MP_EINVAL (n or lda), MP_ENOMEM, MP_ECUDA.
 */
int mp_build_transfer_matrix(int n, int16_t *A, int64_t lda, uint32_t *words_opt,
                             void *stream);

/* ---- a3/a5: one (min,+) product ------------------------------------------
 * Section 1: Z = X (x) Y, Z_ij = min(INF, min_l X_il + Y_lj), exact.
 * X: DEVICE M x K (ldx >= K), Y: DEVICE K x N (ldy >= N), Z: DEVICE M x N
 * (ldz >= N), all of element type dtype (MP_I16 or MP_U8).  K = 0 gives an
 * all-INF Z (X and Y may then be NULL).  M = 0 or N = 0 is a no-op.  Blocks of 128 x 128 that are
 * entirely INF in X or Y are skipped (their terms cannot lower a minimum).
 * An operand whose rows do not start on 8-element boundaries (base address
 * or leading dimension) is repacked into temporary library-owned device
 * memory (M x K or K x N, rows padded to 8) during the mask pass, so every
 * tile is read with 16-byte loads; the caller's arrays are only read.
 * Errors: MP_EINVAL (negative sizes, ld too small, dtype), MP_EALIAS (Z
 * overlaps X or Y), MP_ENOMEM, MP_ECUDA.  Asynchronous.
 */
int mp_minplus_mul(const void *X, const void *Y, void *Z, int64_t M, int64_t N,
                   int64_t K, int64_t ldx, int64_t ldy, int64_t ldz, int dtype,
                   void *stream);

/* The same product for callers that cannot allocate device memory: code
 * running where cudaMalloc is unavailable or forbidden (inside a memory
 * budget owned by another allocator, a real-time path that must not call
 * the allocator, a plugin whose host owns all device memory).  The paper
 * has no counterpart; it is a deployment variant of mp_minplus_mul.
 * It allocates nothing: the only scratch of the product, the per-operand
 * occupancy masks, lives in a fixed 1 MiB device array inside the library
 * that every GPU which loads the library holds until the process exits.
 * Arguments, results and errors as mp_minplus_mul, plus MP_EINVAL when
 * ceil(M/128)*ceil(K/128) + ceil(K/128)*ceil(N/128) exceeds 1048576 (about
 * N = 90000 for square operands).  Unlike mp_minplus_mul, operands whose
 * rows are off the 8-element grid are not repacked (that would need memory):
 * they are read in place with scalar loads, which gives the same result
 * more slowly.  The first call on a device looks up the array's device
 * address with cudaGetSymbolAddress (with that device current); make that
 * first call before any stream capture.  The address is kept per device
 * and looked up again after a cudaDeviceReset.  Every call shares the
 * array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it and must be serialized by the caller. */
int mp_minplus_mul_noalloc(const void *X, const void *Y, void *Z, int64_t M, int64_t N,
                           int64_t K, int64_t ldx, int64_t ldy, int64_t ldz, int dtype,
                           void *stream);

/* ---- a3/a4: the power chain with the gamma_2 readout -----------------------
 * Algorithm 2 and Theorem 2 / Algorithm 5: P_1 = A, P_k = A (x) P_{k-1} for
 * k = 2..k_max (equal to P_{k-1} (x) A by associativity), and
 * g[k-1] = min_i (P_k)_ii.
 * A: DEVICE int16 N x N (leading dimension N), entries in [0, 0x7FFF].
 * powers_opt: DEVICE int16 [k_max][N][N], slot k-1 receives P_k, or NULL
 * (then only two internal ping-pong buffers are used).
 * gdiag_opt: DEVICE int32 [k_max], slot k-1 receives min diag P_k (0x7FFF
 * when the whole diagonal is INF), or NULL.
 * A sparse A (at most 1/4 of its entries finite) runs the sparse transfer
 * kernel; a denser A the dense product.  Synchronizes the stream once to
 * size the sparse plan.  Errors: MP_EINVAL, MP_EALIAS (powers overlap A),
 * MP_ENOMEM, MP_ECUDA.
 */
int mp_minplus_power_sequence(const int16_t *A, int64_t N, int k_max,
                              int16_t *powers_opt, int32_t *gdiag_opt, void *stream);

/* The same chain for the transfer matrix A(D_n) itself, built on the device
 * from n (no dense A is formed).  The plan for n is cached per device after
 * the first call.  powers_opt / gdiag_opt as above with N = |C_n|.
 * Where a column chunk fits shared memory (n <= 9 on GB300) the chain runs
 * on the reuse circuit (mp_transfer_circuit_info) as one launch: each CTA
 * keeps an 8- or 16-column chunk of the powers on chip for every step.
 * Larger n run on the circuit in global memory.  The results are the same
 * bit for bit.  With powers_opt the chain computes only the
 * mirror-representative columns (see below) into a temporary staging area
 * of about k_max * N * N bytes and one copy pass writes every power in full
 * (P_k[R i][R c] = P_k[i][c] for the reversal R); without room for the
 * staging area it computes every column and writes them itself.  A repeated call with the same arguments is replayed from a CUDA
 * graph captured on its second call; a capture that fails (for instance
 * because another host thread synchronised the whole device meanwhile) is
 * dropped and the chain runs directly.
 * With powers_opt NULL the chain computes only one column of every pair
 * {w, reversed w} of column words: reading words backwards is an
 * automorphism of A(D_n), so the dropped columns repeat kept ones, every
 * diagonal value is among the kept columns, and gdiag is the same; the work
 * is about half (a second plan, cached likewise, is built on the first such
 * call).  Synchronizes the stream on the first call of either kind for a
 * given n. */
int mp_transfer_power_sequence(int n, int k_max, int16_t *powers_opt,
                               int32_t *gdiag_opt, void *stream);

/* ---- checkpoint and resume ------------------------------------------------
 * The paper keeps A and its powers on disk between its algorithms
 * (Section 3); a checkpoint lets a long chain stop and resume.  A file holds
 * `count` consecutive powers A^k0 .. A^(k0+count-1) of A(D_n): a 64-byte
 * header ("MPPOWERS", format version 1, n, k0, N, count, the INF code 0x7FFF,
 * the word order -- lexicographic, letter 1 most significant, 0 < 1 < 2 --
 * and a 64-bit FNV-1a hash of the packed word list), then the int16 entries
 * row-major, power after power, little-endian.
 *
 * mp_powers_save: writes DEVICE powers[count][N][N] (slot j = A^(k0+j)).
 * mp_powers_info: HOST only (no CUDA call); writes {n, N, k0, count} into
 *   the HOST array info[0..cap) after checking the header, the word-list
 *   hash and the file size; returns the number of fields written.
 * mp_powers_load: reads every stored power into DEVICE powers (at least
 *   count slots of N x N; cap_slots is the buffer's capacity in slots).
 * mp_transfer_power_sequence_from: Algorithm 2 resumed from a stored power:
 *   given DEVICE P_k0 = A^k0 (N x N, the library's word order), computes
 *   A^(k0+1) .. A^k_max: powers_opt slot j and gdiag_opt[j] receive A^(k0+1+j)
 *   and its minimum diagonal entry (k_max - k0 slots each; either may be
 *   NULL, and without powers the chain runs on the mirror-representative
 *   columns as mp_transfer_power_sequence does).  Bit-identical to the
 *   uninterrupted chain.  Asynchronous apart from one synchronization of the
 *   stream when the plan is first built.
 * save, info and load are synchronous (they wait for stream).  Errors:
 * MP_EINVAL (arguments, a buffer too small), MP_EALIAS, MP_EIO (open, read
 * or write failed; not a checkpoint, another format version, another word
 * list, a size that does not match the header), MP_ENOMEM, MP_ECUDA. */
int mp_powers_save(const char *path, int n, int k0, int64_t count, const int16_t *powers, void *stream);
int mp_powers_info(const char *path, int64_t *info, int cap);
int mp_powers_load(const char *path, int16_t *powers, int64_t cap_slots, void *stream);
int mp_transfer_power_sequence_from(int n, int k0, const int16_t *P_k0, int k_max, int16_t *powers_opt,
                                    int32_t *gdiag_opt, void *stream);

/* ---- a6: gamma_2 of one cylinder --------------------------------------------
 * Theorem 2: gamma_2(P_n x C_m) = min_i (A^m)_ii, for n >= 1 and m >= 3.
 * Synchronous; *out is a HOST int64.  When the recurrence of n is known
 * (mp_transfer_recurrence, run automatically for n <= 11 and m > 64, or
 * mp_transfer_recurrence_stream for larger n) the
 * answer comes from Theorem 3 for any m.  Otherwise it uses the cached
 * transfer plan and either the chain or repeated squaring
 * S_j = S_{j-1} (x) S_{j-1} followed by a min-trace of the last two factors.
 * Errors: MP_EINVAL (n out of range, m < 3), MP_ERANGE (no recurrence and
 * m * n >= 32767: exact values could reach the int16 INF code),
 * MP_ENOMEM, MP_ECUDA.
 */
int mp_gamma2_cylinder(int n, int64_t m, int64_t *out);

/* gamma_2(P_n x C_m) by repeated squaring alone (Theorem 2 with the power
 * algebra of Lemma 1): S_0 = A(D_n), S_j = S_{j-1} (x) S_{j-1} = A^(2^j)
 * (dense products, int16), R = the product of the S_j over the set bits
 * of m below its highest bit t, and *out = min_{i,l} R_il + (S_t)_li, the
 * minimum diagonal entry of A^m, without forming A^m (for m = 2^t,
 * R = S_t = S_{t-1}).  About log2(m) + popcount(m) dense N^3 products, no
 * recurrence and no chain; mp_gamma2_cylinder takes this route itself only
 * when its cost model prefers it.  Needs 4 N^2 * 2 bytes of device memory.
 * Synchronous; *out is a HOST int64.  Errors: MP_EINVAL (n out of range,
 * m < 3, out NULL), MP_ERANGE (m * n >= 32767), MP_ENOMEM, MP_ECUDA. */
int mp_gamma2_squaring(int n, int64_t m, int64_t *out);

/* ---- NEXT f1: the recurrence of Theorem 3 ---------------------------------
 * mp_diff_const (K4): for two DEVICE int16 arrays of count entries, writes to
 * DEVICE int32 out[4]: out[0] = min and out[1] = max of X - Y over the
 * entries finite in both, out[2] = 1 if some entry is INF in exactly one of
 * them (else 0), out[3] = 1 if some entry is finite in both.  X - Y is a
 * constant matrix (Algorithm 3's test, with equal INF patterns) exactly when
 * out[2] == 0, out[3] == 1 and out[0] == out[1].  Asynchronous.
 *
 * mp_transfer_recurrence: Algorithm 3 over K stored powers of A(D_n), then
 * Algorithm 4 (Section 3): out (HOST int32[4]) = {r0, a, b, n0}; a = 0 when
 * no constant difference exists among the K powers.  With K = 50 this is
 * Table 3's (r0, a, b) and Table 4's n0.  Synchronous; needs K*N^2*2 bytes
 * of device memory (MP_ENOMEM otherwise).  A found recurrence is cached per
 * device and used by mp_gamma2_cylinder (Theorem 3), which then answers any
 * m >= 3 without the int16 range limit. */
int mp_diff_const(const int16_t *X, const int16_t *Y, int64_t count, int32_t *out, void *stream);
int mp_transfer_recurrence(int n, int K, int32_t *out);

/* NEXT f2: the same recurrence for path orders whose K powers do not fit:
 * the chain keeps only the last `ring` powers and, after each product P_k,
 * compares P_k with P_{k-a} for a = 1..ring-1 (smallest a first).  The first
 * constant difference, at k = n0 + a, gives Table 4's n0 with a and b.
 * out (HOST int32[4]) = {n0, a, b, k}; a = 0 if nothing is found by k_limit.
 * Synchronous; needs ring*N^2*2 bytes plus two chain buffers (MP_ENOMEM
 * otherwise).  The result is cached for mp_gamma2_cylinder, which runs this
 * form itself (k_limit 64, ring 20) for n >= 12. */
int mp_transfer_recurrence_stream(int n, int k_limit, int ring, int32_t *out);

/* The gamma_2 table of one path order: out[m] = gamma_2(P_n x C_m) for
 * m = 3..k_max (Theorem 2 / Algorithm 5 over the chain), out[0..2] = -1.
 * out is a HOST int64 array of k_max + 1 entries.  Synchronous; runs on a
 * library-owned stream.  Errors: MP_EINVAL (n, k_max < 3), MP_ERANGE
 * (k_max * n >= 32767), MP_ENOMEM, MP_ECUDA. */
int mp_gamma2_table(int n, int k_max, int64_t *out);

/* Several transfer chains at once (Algorithm 2 and Theorem 2 for each path
 * order ns[i], i < count, distinct): gdiag (DEVICE int32, count x k_max,
 * row i for ns[i]) receives min diag A^k for k = 1..k_max as in
 * mp_transfer_power_sequence with powers_opt NULL.  Up to 8 chains that all
 * run on the shared-memory reuse circuit (n <= 9) run in one launch on
 * stream, the longest chain's CTAs first; otherwise the chains run side by
 * side on library-owned streams forked from and joined back into stream.
 * Either way the work is asynchronous on stream and the short chains
 * overlap the long ones.  Errors: MP_EINVAL (count < 0, NULL arrays,
 * k_max < 1, an n out of range or repeated), MP_ENOMEM, MP_ECUDA. */
int mp_transfer_power_sequences(const int *ns, int count, int k_max, int32_t *gdiag,
                                void *stream);

/* The gamma_2 tables of several path orders (HOST int32 ns[count], distinct):
 * out (HOST int64, count x (k_max + 1)) row i holds mp_gamma2_table(ns[i]).
 * Synchronous; the chains run side by side as in mp_transfer_power_sequences.
 * Errors: MP_EINVAL (count < 0, NULL arrays, k_max < 3, an n out of range or
 * repeated), MP_ERANGE (k_max * n >= 32767 for some n), MP_ENOMEM, MP_ECUDA. */
int mp_gamma2_tables(const int *ns, int count, int k_max, int64_t *out);

/* ---- K3: reductions -----------------------------------------------------
 * mp_diag_min: *out = min_i P[i][i] over an N x N DEVICE int16 matrix
 * (leading dimension ld), written to DEVICE int32 out.  Theorem 2.
 * mp_min_trace: *out = min_{i,l} X[i][l] + Y[l][i] (= min diag of X (x) Y
 * without forming it) for N x N DEVICE int16 X, Y; DEVICE int32 out,
 * saturated at 0x7FFF.  Both asynchronous. */
int mp_diag_min(const int16_t *P, int64_t N, int64_t ld, int32_t *out, void *stream);
int mp_min_trace(const int16_t *X, const int16_t *Y, int64_t N, int64_t ldx,
                 int64_t ldy, int32_t *out, void *stream);

/* ---- a7: many products of uneven sizes ----------------------------------------
 * One descriptor per product Z = X (x) Y; pointers are DEVICE, sizes and
 * leading dimensions as for mp_minplus_mul, dtype MP_I16 or MP_U8. */
typedef struct mp_problem {
    const void *X;
    const void *Y;
    void *Z;
    int64_t M, N, K;
    int64_t ldx, ldy, ldz;
    int32_t dtype;
    int32_t reserved;
} mp_problem;

/* Runs every product of probs[0..count) (HOST array).  mode 0: one
 * occupancy-mask launch and one persistent launch over a tile work list of
 * all products; mode 1: a mask launch and a product launch per product (the
 * plain form, for comparison).  No output may overlap any input of any
 * problem.  Prepares, runs and releases a batch (below) and synchronizes
 * the stream before returning.  Errors: MP_EINVAL, MP_EALIAS, MP_ENOMEM,
 * MP_ECUDA. */
int mp_minplus_mul_batched(const mp_problem *probs, int count, int mode, void *stream);

/* A prepared batch: the tile work list (every output tile of every product
 * in the tile shape the tuning table gives its size class, most expensive
 * first), the problem descriptors and the mask-block list are uploaded once
 * (synchronously) and owned by the opaque handle, together with the mask
 * buffer and, for operands whose rows are off the 8-element grid, buffers
 * for their repacked copies (refreshed by every run's mask pass).
 * mp_batch_run only enqueues kernels and one memset on stream, so
 * it may be captured in a CUDA graph and replayed; the operands may change
 * between runs but not their addresses or shapes.  One batch must not run
 * concurrently with itself.  mp_batch_destroy frees the handle (the caller
 * makes sure no run is in flight). */
typedef struct mp_batch mp_batch;
int mp_batch_prepare(const mp_problem *probs, int count, mp_batch **out);
int mp_batch_run(mp_batch *batch, int mode, void *stream);
int mp_batch_destroy(mp_batch *batch);

/* ---- tile-shape autotuner ---------------------------------------------------
 * The dense product uses a 128x128 (shape 0) or 64x64 (shape 1) output
 * tile chosen per element type and size class of min(M, N): [0,128),
 * [128,256), [256,512), [512,1024), [1024,2048), [2048,inf).  The table is
 * int32[2][6] (row 0 int16, row 1 uint8), per device.  mp_autotune times both
 * shapes on one synthetic square product per class on the current device,
 * installs the faster ones and writes the table to table_out (HOST, may be
 * NULL); synchronous.  mp_tuning_set installs a table (e.g. from a cache);
 * mp_tuning_get reads the current one (a built-in default until tuned). */
int mp_autotune(int32_t *table_out);
int mp_tuning_set(const int32_t *table);
int mp_tuning_get(int32_t *table);

/* ---- serving: continuous batching of gamma_2 queries ---------------------
 * A server answers gamma_2(P_n x C_m) (Theorem 2) for a stream of queries.
 * For each path order it serves it keeps powers of A(D_n) resident on the
 * current device: A^1..A^B and, transposed, A^{tB} for t = 1..T, with
 * B = ceil(sqrt(max_m)) and T = ceil(max_m / B).  m <= B is answered from
 * the min-diagonals kept on the host; every larger m <= max_m is one
 * streaming min of A^x + (A^{tB})^T over two resident powers (m = x + tB),
 * read on the rows of one word of every mirror pair only (reading a word
 * backwards is an automorphism of A(D_n), so the other rows repeat the same
 * terms).  A worker thread batches the queries whose path order is
 * resident into one launch (two batches may be in flight); a query for a
 * path order that is not resident admits it: its footprint
 * (B + T) * N^2 * 2 bytes (slots rounded to 8 entries) is checked against hbm_budget, idle path
 * orders are evicted least recently used first, and a builder thread
 * computes the powers on its own stream while other batches run.
 *
 * mp_server_create: hbm_budget in bytes, max_batch queries per launch,
 *   max_m the largest cycle length served, max_tickets the capacity of the
 *   ticket table (the server's lifetime query count).  The server lives on
 *   the current device.
 * mp_server_submit: enqueues (n, m) and returns a ticket; never blocks.
 * mp_server_replay: a load generator: submits query i of the HOST arrays
 *   n[i], m[i] at t_offsets[i] seconds after the call (busy-waiting on a
 *   monotonic clock; t_offsets NULL submits at once), writes the tickets,
 *   and returns once all are submitted (not answered).
 *   MP_EINVAL for n outside [1, 16] or m outside [3, max_m], MP_ERANGE for
 *   m * n >= 32767, MP_EBUSY when the ticket table is full.
 * mp_server_poll: MP_OK with *gamma2 set (HOST int64) once answered,
 *   MP_ENOTREADY before, MP_ENOMEM if the path order can never fit the
 *   budget, MP_EINVAL if the ticket was cancelled or is unknown.
 * mp_server_cancel: withdraws a query not yet answered (MP_EBUSY if it
 *   already was).
 * mp_server_latency: submit and completion times (seconds on a monotonic
 *   clock) of an answered ticket, MP_ENOTREADY before.
 * mp_server_stats: out (HOST int64[8]) = submitted, completed, failed,
 *   cancelled, batches launched, path orders built, evictions, resident bytes.
 * mp_server_destroy: finishes in-flight work, frees everything.
 * Thread safety: submit, poll, cancel, latency and stats may be called from
 * any host thread; create and destroy from one. */
typedef struct mp_server mp_server;
int mp_server_create(size_t hbm_budget, int max_batch, int64_t max_m, int64_t max_tickets,
                     mp_server **out);
int mp_server_submit(mp_server *server, int n, int64_t m, uint64_t *ticket);
int mp_server_replay(mp_server *server, const int32_t *n, const int64_t *m,
                     const double *t_offsets, int64_t count, uint64_t *tickets);
int mp_server_poll(mp_server *server, uint64_t ticket, int64_t *gamma2);
int mp_server_cancel(mp_server *server, uint64_t ticket);
int mp_server_latency(mp_server *server, uint64_t ticket, double *submit_s, double *done_s);
int mp_server_stats(mp_server *server, int64_t *out);
int mp_server_destroy(mp_server *server);

/* ---- K6: DPX add-min peak ------------------------------------------------
 * Runs independent __viaddmin_u16x2 chains on every SM for `iters`
 * iterations and writes the achieved add-min rate (two per instruction) in
 * operations per second to *ops_per_s (HOST).  variant 0: viaddmin u16x2;
 * 1: vimin3 u16x2 (counted as two minima per lane pair); 2: plain vmin u16x2;
 * 3: conflict-free 16-byte shared-memory loads, written as BYTES per second
 * (the roof of the shared-memory-bound transfer step).  Synchronous. */
int mp_dpx_peak(int variant, int64_t iters, double *ops_per_s);

/* ---- failure injection (tests) -------------------------------------------
 * Kernels that wait on the device (the reuse circuit's wait for the bulk
 * copies of its blob) give up after about a second, latch MP_ETIMEOUT in the
 * device status word and return, so a stalled copy cannot hang the GPU.
 * mp_inject_circuit_timeout makes that happen on purpose: it enqueues on
 * stream one step of A(D_n)'s circuit kernel whose wait expects 16 bytes
 * that no copy sends.  Every CTA's wait runs out (about two seconds in all,
 * after the real copies have landed) and the CTA returns without computing
 * or writing anything; the next mp_device_status() returns MP_ETIMEOUT and
 * clears it, and the context stays usable.  The paper has no counterpart.
 * Errors: MP_EINVAL (n out of range or without a circuit), MP_ENOMEM,
 * MP_ECUDA. */
int mp_inject_circuit_timeout(int n, void *stream);

/* ---- device status and errors --------------------------------------------
 * mp_device_status synchronizes the current device, then returns MP_OK or
 * the first latched device-side error (MP_ETIMEOUT; MP_ECHECK in a build
 * compiled with -DMP_CHECK, whose circuit kernels check every shared- and
 * global-memory index they compute, latch MP_ECHECK on one outside its
 * buffer and use index 0 instead, so the access stays in bounds) and clears
 * it. */
int mp_device_status(void);
const char *mp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MINPLUS_H */
