// Sparse (min,+) power-chain plan and launchers (K2).
#pragma once

#include <vector>

#include "mp_internal.cuh"

namespace mp {

#ifdef __CUDACC__
// The 8 values of v (two per word, low half first) to dst[0..8), or only the
// first `valid` of them at the right edge; the caller's rows have any length,
// so the widest store the address allows: one 16-, two 8- or four 4-byte
// stores, or, at an odd address, a 2-byte store, three 4-byte stores of
// re-paired halves and a 2-byte store.
__device__ __forceinline__ void store_row8(int16_t *dst, const uint4 &v, int64_t valid) {
    const uintptr_t ad = (uintptr_t)dst;
    if (valid >= 8) {
        if ((ad & 15) == 0) {
            *reinterpret_cast<uint4 *>(dst) = v;
        } else if ((ad & 7) == 0) {
            reinterpret_cast<uint2 *>(dst)[0] = make_uint2(v.x, v.y);
            reinterpret_cast<uint2 *>(dst)[1] = make_uint2(v.z, v.w);
        } else if ((ad & 3) == 0) {
            uint32_t *d = reinterpret_cast<uint32_t *>(dst);
            d[0] = v.x;
            d[1] = v.y;
            d[2] = v.z;
            d[3] = v.w;
        } else {
            dst[0] = (int16_t)(v.x & 0xFFFFu);
            uint32_t *d = reinterpret_cast<uint32_t *>(dst + 1);
            d[0] = __byte_perm(v.x, v.y, 0x5432);
            d[1] = __byte_perm(v.y, v.z, 0x5432);
            d[2] = __byte_perm(v.z, v.w, 0x5432);
            dst[7] = (int16_t)(v.w >> 16);
        }
        return;
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const uint32_t wv = kk < 2 ? v.x : kk < 4 ? v.y : kk < 6 ? v.z : v.w;
        if (kk < valid) dst[kk] = (int16_t)((kk & 1) ? wv >> 16 : wv & 0xFFFFu);
    }
}

#endif

// Shape of the sparse step shared by the kernel (spmm.cu) and the host plan
// builder (spmm_plan.cu).
constexpr int kThreads = 512;                    // 16 warps
constexpr int kWarps = kThreads / 32;
constexpr int kGroupMax = 64;                     // rows per group (6-bit row indices)
constexpr int kChunk = 64;                        // columns per work item
constexpr int kRowBytes = kChunk * 2;
constexpr int kBlobHeader = 48;  // words: row0, nrows, flags, ntasks, nsegs, 3 pad, per-warp task
                                 // starts (kWarps + 1), per-warp stream starts (kWarps + 1)
constexpr int kAccBytes = kGroupMax * kChunk * 4;  // per-row accumulators, one word per column
constexpr int kStageRowsMax = 768;                // U rows per stage (register-staged indices)
constexpr int kStagesMax = 3;                     // stages per group when rows are long
constexpr int kRowLoads = kStageRowsMax * (kRowBytes / 16) / kThreads;  // 12 per thread

// Entry words of the column-constant stream: bits 0..16 the byte offset of
// the gathered row in the row buffer.  A segment is a whole number of 8-entry
// pairs of 4-entry blocks; every entry of its last block has bit 31 set and
// bits 17..20 = the segment's cluster mask, and bit 30 too when the block
// also ends a task.
constexpr uint32_t kEntOffset = 0x1FFFFu;
constexpr uint32_t kEntSegEnd = 0x80000000u;
constexpr uint32_t kEntTaskEnd = 0x40000000u;
constexpr int kEntMaskShift = 17;
constexpr int kStreamStart = 8 + kWarps + 1;  // header words: per-warp stream starts
static_assert(kStreamStart + kWarps < kBlobHeader, "blob header too small");

// CSR of a sparse N x N int16 matrix: the finite entries of each row.
struct HostCsr {
    int64_t N = 0;
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col;
    std::vector<int16_t> val;
};
struct DevCsr {
    DevBuf row_ptr, col, val;
};

// One unit of a CTA's schedule: stage s of work item (group, chunk), packed
// into 16 bytes: meta = chunk (bits 0-15) | blob words / 8 (bits 16-30) |
// last stage of its item (bit 31); u0, u1 = the stage's rows in urows;
// bo8 = blob offset in 8-word granules.
struct UnitDesc {
    uint32_t meta, u0, u1, bo8;
};

// The gather plan of a sparse A, built once on the host (spmm_plan.cu).
struct PlanHost {
    int64_t N = 0, ldb = 0, nnz = 0;
    int ngroups = 0, nchunks = 0, cap_rows = 0, blob_cap = 0;
    bool colconst = false;
    std::vector<int32_t> grp_row0, grp_stage0, stage_u0, urows;
    std::vector<int64_t> blob_off;
    std::vector<uint32_t> blob;
    std::vector<uint16_t> z;
    int grid = 0;                         // CTAs the schedule is made for
    std::vector<UnitDesc> units;          // every CTA's units, back to back
    std::vector<int32_t> cta_unit0;       // [grid + 1] offsets into units
    // The chain may keep the rows of its powers in an order of its own
    // (rows of the plan = rows of the internal buffers): canon[i] is the row
    // (and diagonal column) of the caller's matrices that internal row i
    // holds.  Empty: the identity.  Columns are never reordered.
    std::vector<int32_t> canon;
    // A narrow chain keeps only some columns: colpos[c] is the buffer column
    // of caller column c, or -1.  Empty: all columns, in the caller's order.
    std::vector<int32_t> colpos;
};
// The reuse circuit of a column-constant sparse A (circuit.cu).  Row q of
// A (x) X is the minimum, over the rows p with an arc q -> p, of z_p + X[p];
// when the arcs out of q' are a subset of those out of q, that minimum over
// q' is a part of q's, so row q is the minimum of a few rows of the result
// itself (its cover) and of the rows X[p] the cover leaves out.  Rows are
// computed in levels (a row after every row of its cover), one column chunk
// of 8 columns per CTA with the chunk of X, of the result and the circuit
// itself in shared memory.
struct CircuitCover {
    int64_t N = 0;
    int levels = 0;
    // per row its list: rows of X (p < N) and rows of the result (N + q')
    std::vector<std::vector<uint32_t>> lists;
    std::vector<int> level;
    int64_t reads = 0, cover_reads = 0;  // list entries, of them result rows
};
// Columns per CTA chunk: a row of the chunk is 16 bytes, one lane's load.
constexpr int kCircW = 8;
// Rows of one lane task: a list of up to 8 image rows; a row with a longer
// list takes 2, 4, ... 32 lanes (an aligned group), whose partial minima a
// warp combines by shuffles.
constexpr int kCircLaneMax = 32;
// A cover candidate must save more than kCircLambda row reads for each level
// it adds to its row: fewer, fuller levels for a few more reads.
constexpr int kCircLambda = 4;
struct CircuitHost {
    int64_t N = 0;
    int64_t Nh = 0;  // N rounded up to 8: the result rows start at image row Nh
    int W = 0, levels = 0;
    std::vector<int32_t> level_slice0;  // [levels + 1] first warp slice of each level
    // per lane task, 32 per warp slice: info = row | log2(lanes of its row)
    // << 16 (row 0xFFFF: an idle lane), and a block of 8 image-row indices
    // (X rows 0..N-1, result rows Nh..Nh+N-1; 2Nh, the INF row, pads)
    std::vector<uint32_t> info;
    std::vector<uint16_t> ents;
    int64_t reads = 0, cover_reads = 0;  // row reads of the circuit, of them result rows
    int64_t lanes = 0;                   // lane tasks that hold a row
};
struct CircuitDev {
    int W = 0, levels = 0;
    int64_t Nh = 0;
    int64_t nslices = 0;
    // the circuit as one blob, copied whole into shared memory: level
    // starts, lane infos, lane entry blocks, the rows' labels
    DevBuf meta;
    uint32_t meta_bytes = 0, off_info = 0, off_ents = 0, off_z = 0;
    DevBuf drow;    // per buffer column: the internal row whose diagonal entry it holds (0xFFFF: none)
    DevBuf caller;  // per internal row: the caller's row (int32), for writing full powers
    bool ready = false;
};

// The circuit of a path order whose chunk does not fit shared memory
// (gcircuit.cu): per level, warp tasks of 32 / L rows, each row slot
// {row, first entry / 4, entries / 4, the task's longest list / 4}; entry
// words: the row in bits 0..23, bit 31 for a result row (a cover), bit 30
// for padding, the label of a direct read in bits 24..27.
struct GCircuitHost {
    int64_t N = 0;
    int L = 0, levels = 0;  // lanes per row: chunks of 8 L columns
    std::vector<uint32_t> level_task0;
    struct Slot {
        uint32_t row, off4, len4, tmax4;
    };
    std::vector<Slot> tasks;
    std::vector<uint32_t> ents;
    int64_t reads = 0, cover_reads = 0;
};
struct GCircuitDev {
    int L = 0, levels = 0;
    int64_t reads = 0, cover_reads = 0;
    size_t bytes = 0;
    DevBuf level_task0, tasks, ents;
    DevBuf drow;    // per buffer column: the internal row with its diagonal entry there (uint32)
    DevBuf caller;  // per internal row: the caller's row (int32)
    bool ready = false;
};

struct PlanDev {
    int64_t N = 0, ldb = 0, nnz = 0;
    int ngroups = 0, nchunks = 0, cap_rows = 0, blob_cap = 0;
    bool colconst = false;
    size_t h2d_bytes = 0;
    int grid = 0;
    DevBuf grp_row0, grp_stage0, stage_u0, blob_off, blob, uoff16, z, units, cta_unit0;
    DevBuf canon;          // empty: identity row order
    bool permuted = false;
    DevBuf colpos;         // empty: all columns
    bool narrow = false;
    CircuitDev circuit;    // used for the steps when ready
    GCircuitDev gcircuit;  // used for the steps when ready; its buffers hold unlabelled powers
};

// Whether a plan's chain buffers hold z_q + P[q] (the gather plan and the
// shared-memory circuit) or P itself (the global circuit).
inline bool plan_labelled(const PlanDev &p) { return p.colconst && !p.gcircuit.ready; }

struct SpStepArgs {
    const uint32_t *uoff16;  // gathered rows: offsets into Bin in 16-byte units
    const uint32_t *blob;
    const UnitDesc *units;
    const int32_t *cta_unit0;
    int cap_rows, blob_cap;
    int64_t N, ldb;
    const uint16_t *Bin;
    uint16_t *Bout;
    int16_t *user_out;
    int32_t *gdiag;
    int *status;
};

// canon: per row, the word written to the blob (the caller row, which is also
// the buffer column of the row's diagonal entry), NULL for the identity;
// ncols: columns of the chain's buffers (<= 0: N).
int plan_build_host(const HostCsr &csr, bool colconst, const std::vector<uint16_t> &z,
                    const std::vector<int32_t> *canon, int64_t ncols, int cap_rows, int blob_cap,
                    int grid, PlanHost *out, int cluster_max = 4);
int plan_upload(const PlanHost &h, PlanDev *d, cudaStream_t s, bool persistent);
int sparse_cap_rows(int *cap_rows, int *blob_cap, int *grid);
int sparse_step(const PlanDev &p, const uint16_t *Bin, uint16_t *Bout, int16_t *user_out,
                int32_t *gdiag, cudaStream_t s);
int sparse_init_from_dense(const PlanDev &p, const int16_t *A, uint16_t *B0, int16_t *user0,
                           int32_t *g0, cudaStream_t s);
int sparse_init_from_csr(const PlanDev &p, const int64_t *row_ptr, const int32_t *col,
                         const int16_t *val, uint16_t *B0, int16_t *user0, int32_t *g0,
                         cudaStream_t s);
// The same for a block of `width` buffer columns from col_base (B0 holds
// only the block, width columns per row).
int sparse_init_block_from_csr(const PlanDev &p, const int64_t *row_ptr, const int32_t *col,
                               const int16_t *val, int64_t col_base, int64_t width, uint16_t *B0,
                               int32_t *g0, cudaStream_t s);
int dense_to_csr(const int16_t *A, int64_t N, HostCsr *csr, DevCsr *dcsr, cudaStream_t s);
// B0 = the labelled buffer of a caller's power P (N x N, caller rows and
// columns): internal row q holds z_q + P[canon[q]][colmap[j]] at buffer
// column j < ncols (colmap NULL: j itself), z_q + INF beyond.
int sparse_init_from_power(const PlanDev &p, const int16_t *P, const int32_t *colmap, int64_t ncols,
                           uint16_t *B0, cudaStream_t s);

// The covers and levels of a column-constant CSR (a row's arcs may not
// repeat; lambda: cover reads given up per level saved), and their slicing
// into lane tasks.
int circuit_cover_host(const HostCsr &csr, CircuitCover *out, int lambda = kCircLambda);
int circuit_slice_host(const CircuitCover &cv, CircuitHost *out);
int circuit_build_host(const HostCsr &csr, CircuitHost *out);
// Shared memory a step takes with this circuit (0: too large for the device).
int circuit_smem_bytes(const CircuitHost &h, size_t *bytes);
// Attach a circuit to a plan: z = the rows' labels, diagcol[q] = the buffer
// column of internal row q's diagonal entry or -1, caller[q] = the caller's
// row of internal row q.
int circuit_upload(const CircuitHost &h, const std::vector<uint16_t> &z,
                   const std::vector<int32_t> &diagcol, const std::vector<int32_t> &caller,
                   PlanDev *d, cudaStream_t s);
int circuit_step(const PlanDev &p, const uint16_t *Bin, uint16_t *Bout, int16_t *user_out,
                 int32_t *gdiag, cudaStream_t s);
// The whole chain P_2 .. P_{k_max} from B1 (the labelled buffer of P_1) in
// one launch: each CTA keeps its column chunk in shared memory from step to
// step.  powers (optional): P_k at powers + (k - 1) * slot in the caller's
// layout; gdiag (optional): g[k - 1] = min diag P_k, folded by atomicMin.
// out_k0: P_k goes to powers slot k - out_k0 and gdiag[k - out_k0] (1 for a
// chain from A itself).  powers_ld: entries between the rows of a power (0:
// N; a multiple of 8 no smaller than the buffer's width makes every row piece
// one aligned 16-byte store, the entries past N left as they come).
int circuit_chain(const PlanDev &p, const uint16_t *B1, int k_max, int16_t *powers, size_t slot,
                  int32_t *gdiag, cudaStream_t s, int out_k0 = 1, int64_t powers_ld = 0);
// count N x N powers from rows of src_ld entries (src_slot between powers) to
// rows of N entries (dst_slot between powers), one launch.
int launch_repack_powers(const int16_t *src, int64_t src_ld, size_t src_slot, int16_t *dst, size_t dst_slot,
                         int64_t N, int count, cudaStream_t s);
// A chain staging its powers chunk by chunk (P_k in stage slot k - 1, slot
// >= N x ldb entries): each power is ldb / W chunks of N rows (internal
// order) of W entries, written by the label pass; *width receives W.
int circuit_chain_staged(const PlanDev &p, const uint16_t *B1, int k_max, int16_t *stage, size_t slot,
                         int32_t *gdiag, cudaStream_t s, int *width);
// count N x N powers from a narrow chain's chunk-major staging (chunks of W
// buffer columns, N internal rows each, src_slot between powers): caller row
// i, column c of power k is internal row inv[i], buffer column mcol[c], or,
// where mcol[c] has bit 31 set, internal row inv[mrow[i]], buffer column
// mcol[c] & 0x7FFFFFFF (the reversal symmetry).  lead[0 .. nlead) are the
// rows i <= mrow[i]: each pair {i, mrow[i]} is written from its two staged
// rows, read once.  One launch.
int launch_mirror_repack(const int16_t *src, int W, int64_t ldb, size_t src_slot, int16_t *dst, size_t dst_slot,
                         const int32_t *mcol, const int32_t *mrow, const int32_t *inv, const int32_t *lead,
                         int64_t nlead, int64_t N, int count, cudaStream_t s);
// The global circuit (n >= 10): covers from the arc rule (words: the
// caller's packed words; canon: internal row -> word), its warp tasks for
// chunks of 8 L columns (z: labels of the internal rows), and the steps.
int circuit_cover_structured(int n, const std::vector<uint32_t> &words, const std::vector<int32_t> &canon,
                             const HostCsr &csr, int lambda, CircuitCover *out);
int gcircuit_slice_host(const CircuitCover &cv, const std::vector<uint16_t> &z, int L, GCircuitHost *out);
int gcircuit_upload(const GCircuitHost &h, const std::vector<int32_t> &diagcol, const std::vector<int32_t> &caller,
                    PlanDev *d, cudaStream_t s);
int gcircuit_step(const PlanDev &p, const uint16_t *Bin, uint16_t *Bout, int16_t *user_out, int32_t *gdiag,
                  cudaStream_t s);
int gcircuit_chain(const PlanDev &p, uint16_t *B0, uint16_t *B1, int k_max, int16_t *powers, size_t slot,
                   int32_t *gdiag, cudaStream_t s, int out_k0 = 1);
// The same on a block of `width` plan columns from col_base (both multiples
// of the chunk): the buffers hold only the block, width columns per row.
int gcircuit_block_step(const PlanDev &p, const uint16_t *Bin, uint16_t *Bout, int64_t col_base, int64_t width,
                        int32_t *gdiag, cudaStream_t s);
int gcircuit_block_chain(const PlanDev &p, uint16_t *B0, uint16_t *B1, int k_max, int64_t col_base,
                         int64_t width, int32_t *gdiag, cudaStream_t s);
int gcircuit_chunk(const PlanDev &p);  // columns per chunk (0: no global circuit)

// Several chains (at most 8, each plan with a circuit) in one launch, the
// CTAs of plans[0] first: B1[i] the labelled buffer of chain i's P_1, gdiag[i]
// its diagonal minima.
int circuit_multi_chain(const PlanDev *const *plans, const uint16_t *const *B1, int count, int k_max,
                        int32_t *const *gdiag, cudaStream_t s);

// Failure injection: one step whose bounded wait for the circuit's copies
// runs out (MP_ETIMEOUT latched in the device status word, nothing written).
int circuit_timeout_probe(const PlanDev &p, const uint16_t *Bin, uint16_t *Bout, cudaStream_t s);

}  // namespace mp
