// K2: the (min,+) power chain over a sparse matrix (Algorithm 2).
//
// P_k = A (x) P_{k-1}: row q of P_k is min over the finite entries A[q][p]
// of A[q][p] + P_{k-1}[p][:], so each output row gathers whole rows of the
// previous power.  The powers are dense from the third one on (Section 3)
// while A stays sparse, so a step costs N * nnz(A) add-min terms instead of
// N^3.  For the transfer matrix every arc into p has the same label z_p,
// the number of zeros of word p (Section 2.2); the kernel then keeps
// B_k[p][:] = z_p + P_k[p][:] between steps (the label pre-added when a row
// is written) and the gather needs only minima, two per instruction with
// __vimin3_u16x2.  Any other sparse A takes per-entry __viaddmin_u16x2.
//
// Work decomposition.  Output rows are grouped greedily (consecutive rows,
// at most 64) so that the union U of the rows they gather fits one shared
// buffer; the columns are cut into chunks of 64.  A work item is (group,
// chunk); a U list longer than one buffer is cut into stages whose per-row
// minima carry over in shared accumulators.  A persistent CTA (one per SM,
// 16 warps) walks its schedule of units (a stage of an item) through two
// shared-memory buffers: while it computes one unit, all threads stream the
// next into the other buffer with 16-byte cp.async copies -- the 128-byte
// segments of the U rows (from 32-bit row offsets precomputed on the host)
// and one "blob" with the unit's task table, row labels and entry streams.
//
// Column-constant A (the transfer matrix).  Rows of a group are clustered
// (up to four rows whose gather lists overlap most); a cluster's union is
// split by membership mask into segments, so every gathered row of a
// segment feeds the same cluster rows.  A segment is reduced once and its
// minimum folded into the rows its mask names: rows that share a gathered
// row share its read and its min.  The unit's clusters, laid out one after
// another, are cut into 16 contiguous ranges of equal modelled cost, one per
// warp; a cluster cut in two becomes two tasks.  Each warp walks its range as
// one stream of entry words (row offset plus segment and task flags); its
// four quarter-warps take one entry each, so one 16-byte shared load per
// lane reads four gathered rows.  At a task end the quarters' minima are
// combined with shuffles and folded into the rows' shared accumulators with
// atomicMin; after the last stage of an item one pass writes the rows out.
// A general sparse A keeps one row per task and per-entry labels.
// (1-D TMA bulk copies were tried first for the row segments: at 128 bytes
// each they issued far too slowly to feed the arithmetic.)
// Rows of the next power go to a padded internal buffer (and, when asked,
// to the caller's power array); the diagonal entries are min-reduced in
// registers and folded into g[k] with one atomicMin per warp.  Steps are
// chained with programmatic dependent launch: a step's prologue (reading
// only the plan) overlaps the previous step's tail.
#include <algorithm>
#include <cstring>
#include <iterator>

#include "mp_internal.cuh"
#include "spmm.cuh"

namespace mp {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ uint32_t lds32(const uint8_t *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}

__device__ __forceinline__ void cp_async16_sh(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint4 lds_v4(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr));
    return v;
}

// Row offsets of one unit (in 16-byte units of the input power), one
// register per 16-byte piece this thread copies; ~0u where there is none.
struct RowIdx {
    uint32_t r[kRowLoads];
};

__device__ __forceinline__ void load_row_idx(const SpStepArgs &a, const UnitDesc &u, RowIdx &ri) {
    const int nu = (int)(u.u1 - u.u0);
    const uint32_t *src = a.uoff16 + u.u0 + (threadIdx.x >> 3);
#pragma unroll
    for (int j = 0; j < kRowLoads; ++j)
        ri.r[j] = (int)(threadIdx.x >> 3) + j * (kThreads / 8) < nu ? __ldg(src + j * (kThreads / 8))
                                                                     : 0xFFFFFFFFu;
}

__device__ __forceinline__ int unit_chunk(const UnitDesc &u) { return (int)(u.meta & 0xFFFFu); }
__device__ __forceinline__ bool unit_last(const UnitDesc &u) { return (u.meta >> 31) != 0; }
__device__ __forceinline__ int unit_bw(const UnitDesc &u) { return (int)((u.meta >> 16) & 0x7FFFu) * 8; }

// All threads stream one unit into buf: its blob, then the 64-column
// segments of its gathered rows (offsets already in registers).  Thread t
// copies piece t % 8 of rows t / 8, t / 8 + 64, ...
__device__ __forceinline__ void stage_in(const SpStepArgs &a, const UnitDesc &u,
                                         const RowIdx &ri, uint8_t *buf, size_t blob_bytes) {
    const int tid = threadIdx.x;
    const uint32_t *bsrc = a.blob + (size_t)u.bo8 * 8;
    const int bchunks = unit_bw(u) >> 2;
    for (int c = tid; c < bchunks; c += kThreads) cp_async16(buf + (size_t)c * 16, bsrc + 4 * c);
    const uint4 *base = reinterpret_cast<const uint4 *>(a.Bin + (int64_t)unit_chunk(u) * kChunk) + (tid & 7);
    const uint32_t dst = smem_u32(buf + blob_bytes) + (uint32_t)(tid >> 3) * kRowBytes + (tid & 7) * 16;
#pragma unroll
    for (int j = 0; j < kRowLoads; ++j)
        if (ri.r[j] != 0xFFFFFFFFu)
            cp_async16_sh(dst + (uint32_t)j * (kThreads / 8) * kRowBytes, base + ri.r[j]);
}

// Descriptor k of this CTA, or an empty one (u0 = u1 = 0xFFFFFFFF) past the end.
__device__ __forceinline__ UnitDesc load_unit(const SpStepArgs &a, int k, int k_end) {
    if (k < k_end) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(a.units) + k);
        return UnitDesc{v.x, v.y, v.z, v.w};
    }
    return UnitDesc{0u, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u};
}
__device__ __forceinline__ bool unit_valid(const UnitDesc &u) { return u.u0 != 0xFFFFFFFFu; }

// Lane layout of the stream: quarter qd = lane / 8 takes entry qd of every
// 4-entry block, and lane l8 = lane % 8 of the quarter holds bytes
// 16 l8 .. 16 l8 + 15 of the gathered row (columns 8 l8 .. 8 l8 + 7, two per
// 32-bit word).  One 16-byte shared load per lane reads four gathered rows.

// The four quarters' minima of one cluster row, reduced and scattered so
// that lane (qd, l8) ends with word qd: columns 8 l8 + 2 qd and + 1.
__device__ __forceinline__ uint32_t quarter_reduce(const uint32_t (&x)[4], int qd) {
    const bool hi = qd >= 2;
    uint32_t k0 = hi ? x[2] : x[0], k1 = hi ? x[3] : x[1];
    const uint32_t y0 = hi ? x[0] : x[2], y1 = hi ? x[1] : x[3];
    k0 = __vminu2(k0, __shfl_xor_sync(0xFFFFFFFFu, y0, 16));
    k1 = __vminu2(k1, __shfl_xor_sync(0xFFFFFFFFu, y1, 16));
    const bool odd = qd & 1;
    const uint32_t k = odd ? k1 : k0, y = odd ? k0 : k1;
    return __vminu2(k, __shfl_xor_sync(0xFFFFFFFFu, y, 8));
}

// Cluster rows of a finished task into the shared accumulators: the four
// quarters' minima are reduced, then two 16-bit atomic minima per lane.
template <int NR>
__device__ __forceinline__ void task_flush(uint32_t t0, uint32_t (&m)[4][4], uint32_t *accs,
                                           int qd, int l8) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const uint32_t x = quarter_reduce(m[j], qd);
        uint32_t *acc = accs + (int)((t0 >> (6 * j)) & 0x3Fu) * kChunk + 8 * l8 + 2 * qd;
        atomicMin(acc, x & 0xFFFFu);
        atomicMin(acc + 1, x >> 16);
#pragma unroll
        for (int k = 0; k < 4; ++k) m[j][k] = 0xFFFFFFFFu;
    }
}

// At a segment end: fold the segment minimum s into the cluster rows its mask
// names; at a task end also fold the cluster rows into the shared
// accumulators.  Flags and masks are the same in all four entries of a
// block, so every branch here is warp-uniform.
__device__ __forceinline__ void seg_end(uint32_t w, uint32_t (&s)[4], uint32_t (&m)[4][4],
                                        uint32_t *accs, const uint32_t *tasks, int &t, int qd,
                                        int l8) {
    const uint32_t mask = w >> kEntMaskShift;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (mask & (1u << j)) {
#pragma unroll
            for (int k = 0; k < 4; ++k) m[j][k] = __vminu2(m[j][k], s[k]);
        }
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] = 0xFFFFFFFFu;
    if (w & kEntTaskEnd) {
        const uint32_t t0 = tasks[t++];
        const uint32_t nr = t0 >> 24;
        if (nr == 1) task_flush<1>(t0, m, accs, qd, l8);
        else if (nr == 2) task_flush<2>(t0, m, accs, qd, l8);
        else if (nr == 3) task_flush<3>(t0, m, accs, qd, l8);
        else task_flush<4>(t0, m, accs, qd, l8);
    }
}

// One warp's share of a unit, as one stream of entries [e, e_end).  A
// segment is a whole number of 8-entry pairs of blocks and only the second
// block of a pair can end one, so the inner loop is a tight pass over pairs
// that exits on that flag.  Every entry of a segment feeds the same cluster
// rows, so the segment is reduced once (__vimin3_u16x2, two blocks per
// instruction) and folded into its rows at the segment end: the DPX work per
// entry does not grow with the rows that share it.  The next pair's entry
// words are read while the current pair's rows are loaded.
__device__ __forceinline__ void warp_stream(uint32_t *accs, uint32_t ents_sh, uint32_t rows_sh,
                                            const uint32_t *tasks, int e, int e_end, int t,
                                            int lane) {
    if (e >= e_end) return;
    const int qd = lane >> 3, l8 = lane & 7;
    const uint32_t ib = ents_sh + 4 * qd;  // this quarter's entry of a block
    const uint32_t rb = rows_sh + 16 * l8;  // this lane's 16 bytes of a gathered row
    uint32_t m[4][4], s[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        s[k] = 0xFFFFFFFFu;
#pragma unroll
        for (int j = 0; j < 4; ++j) m[j][k] = 0xFFFFFFFFu;
    }
    uint32_t w0 = lds_u32(ib + 4 * e), w1 = lds_u32(ib + 4 * e + 16);
    do {
        uint32_t f;
        do {
            const uint4 d0 = lds_v4(rb + w0);  // first blocks of pairs carry no flags
            const uint4 d1 = lds_v4(rb + (w1 & kEntOffset));
            f = w1;
            e += 8;
            const int en = min(e, e_end - 8);  // past the end: re-read the last pair
            w0 = lds_u32(ib + 4 * en);
            w1 = lds_u32(ib + 4 * en + 16);
            s[0] = __vimin3_u16x2(s[0], d0.x, d1.x);
            s[1] = __vimin3_u16x2(s[1], d0.y, d1.y);
            s[2] = __vimin3_u16x2(s[2], d0.z, d1.z);
            s[3] = __vimin3_u16x2(s[3], d0.w, d1.w);
        } while (!(f & kEntSegEnd));
        seg_end(f, s, m, accs, tasks, t, qd, l8);
    } while (e < e_end);
}

template <bool kColConst>
__global__ void __launch_bounds__(kThreads, 1) sparse_step_kernel(SpStepArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const size_t blob_bytes = (size_t)a.blob_cap * 4;
    const size_t buf_bytes = blob_bytes + (size_t)a.cap_rows * kRowBytes;
    uint32_t *accs = reinterpret_cast<uint32_t *>(smem + 2 * buf_bytes);  // [64 rows][64 cols]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // the last gathered row of each buffer is the padding row: above any value
    if (threadIdx.x < 64) {
        uint8_t *infrow = smem + (threadIdx.x >> 5) * buf_bytes + blob_bytes +
                          (size_t)(a.cap_rows - 1) * kRowBytes;
        reinterpret_cast<uint32_t *>(infrow)[lane] = 0xFFFFFFFFu;
    }
    for (int i = threadIdx.x; i < kGroupMax * kChunk; i += kThreads) accs[i] = kInf16;

    // this CTA's units, in order; descriptors run two units ahead of the
    // copies and row indices one unit ahead, so no unit waits on a global load
    const int k0 = a.cta_unit0[blockIdx.x], k_end = a.cta_unit0[blockIdx.x + 1];
    if (k0 >= k_end) return;
    UnitDesc cur = load_unit(a, k0, k_end);
    RowIdx idx;
    load_row_idx(a, cur, idx);
    // Programmatic dependent launch: everything above reads only the plan;
    // the previous step's output (our input, and the buffer we overwrite)
    // is touched only after its grid has completed.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    stage_in(a, cur, idx, smem, blob_bytes);
    cp_async_commit();
    UnitDesc nxt = load_unit(a, k0 + 1, k_end);
    if (unit_valid(nxt)) load_row_idx(a, nxt, idx);
    UnitDesc nxt2 = load_unit(a, k0 + 2, k_end);

    int32_t dmin = (int32_t)kInf16;
    for (int k = k0; k < k_end; ++k) {
        const int b = (k - k0) & 1;
        // one barrier per unit: after it this unit's copies are visible to
        // all threads and every warp is done with the previous unit, so its
        // buffer takes the next unit's copies while this one is computed
        cp_async_wait<0>();
        __syncthreads();
        if (unit_valid(nxt)) {
            stage_in(a, nxt, idx, smem + (b ^ 1) * buf_bytes, blob_bytes);
            cp_async_commit();
            if (unit_valid(nxt2)) load_row_idx(a, nxt2, idx);
        }
        const UnitDesc nxt3 = load_unit(a, k + 3, k_end);

        const uint8_t *buf = smem + b * buf_bytes;
        const uint32_t *blob = reinterpret_cast<const uint32_t *>(buf);
        const int row0 = (int)blob[0], nrows = (int)blob[1];
        const int ntasks = (int)blob[3], nsegs = (int)blob[4];
        const uint32_t *tasks = blob + kBlobHeader;
        const uint8_t *sb = buf + blob_bytes + lane * 4;
        const int64_t c0 = (int64_t)unit_chunk(cur) * kChunk;
        const uint16_t *zs;
        if (kColConst) {
            // one task word per task, the labels, then every warp's entry
            // stream (sixteen-byte aligned, a whole number of 8-entry blocks)
            zs = reinterpret_cast<const uint16_t *>(tasks + ((ntasks + 7) & ~7));
            const uint32_t *ents = reinterpret_cast<const uint32_t *>(zs) + ((nrows + 15) / 16) * 8 +
                                   ((nrows + 7) & ~7);
            warp_stream(accs, smem_u32(ents), smem_u32(buf + blob_bytes), tasks,
                        (int)blob[kStreamStart + warp], (int)blob[kStreamStart + warp + 1],
                        (int)blob[8 + warp], lane);
        } else {
            const uint32_t *segs = tasks + ((2 * ntasks + 7) & ~7);
            zs = reinterpret_cast<const uint16_t *>(segs + ((2 * nsegs + 7) & ~7));
            const uint32_t *ents = reinterpret_cast<const uint32_t *>(zs) + ((nrows + 15) / 16) * 8 +
                                   ((nrows + 7) & ~7);
            const int t_end = (int)blob[8 + warp + 1];
            for (int t = (int)blob[8 + warp]; t < t_end; ++t) {
                const uint32_t t0 = tasks[2 * t], t1 = tasks[2 * t + 1];
                uint32_t mm = 0xFFFFFFFFu;
                for (int sg = (int)(t1 & 0xFFFFu); sg < (int)(t1 >> 16); ++sg) {
                    const int e0 = (int)(segs[2 * sg] & 0xFFFFu), e1 = (int)segs[2 * sg + 1];
                    // two entries (offset, label pair) per 16-byte read, four per iteration
#pragma unroll 2
                    for (int e = e0; e < e1; e += 8) {
                        const uint4 p = *reinterpret_cast<const uint4 *>(ents + e);
                        const uint4 q = *reinterpret_cast<const uint4 *>(ents + e + 4);
                        mm = __viaddmin_u16x2(lds32(sb + p.x), p.y, mm);
                        mm = __viaddmin_u16x2(lds32(sb + p.z), p.w, mm);
                        mm = __viaddmin_u16x2(lds32(sb + q.x), q.y, mm);
                        mm = __viaddmin_u16x2(lds32(sb + q.z), q.w, mm);
                    }
                }
                uint32_t *acc = accs + (int)(t0 & 0x3Fu) * kChunk + 2 * lane;
                atomicMin(acc, mm & 0xFFFFu);
                atomicMin(acc + 1, mm >> 16);
            }
        }
        if (unit_last(cur)) {
            __syncthreads();
            // write the item's rows: min(INF, .) since the accumulators start at INF
            const bool diag = a.gdiag != nullptr;
            for (int r = warp; r < nrows; r += kWarps) {
                uint2 *acc = reinterpret_cast<uint2 *>(accs + r * kChunk + 2 * lane);
                const uint2 av = *acc;
                *acc = make_uint2(kInf16, kInf16);
                const uint32_t v = av.x | (av.y << 16);
                const int64_t q = row0 + r;
                const uint32_t keep = kColConst ? v + (uint32_t)zs[r] * 0x10001u : v;
                uint16_t *brow = a.Bout + q * a.ldb + c0;
                reinterpret_cast<uint32_t *>(brow)[lane] = keep;
                // the caller's row (and diagonal column) of internal row q,
                // from the blob (after the labels)
                const int64_t qc = (int64_t)reinterpret_cast<const uint32_t *>(zs)[((nrows + 15) / 16) * 8 + r];
                if (a.user_out) {
                    const int64_t c = c0 + 2 * lane;
                    int16_t *orow = a.user_out + qc * a.N;
                    if (c < a.N) orow[c] = (int16_t)(v & 0xFFFFu);
                    if (c + 1 < a.N) orow[c + 1] = (int16_t)(v >> 16);
                }
                if (diag && qc >= c0 && qc < c0 + kChunk && (int)(qc - c0) >> 1 == lane)
                    dmin = min(dmin, (int32_t)((qc - c0) & 1 ? v >> 16 : v & 0xFFFFu));
            }
        }
        cur = nxt;
        nxt = nxt2;
        nxt2 = nxt3;
    }
    if (a.gdiag) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dmin = min(dmin, __shfl_xor_sync(0xFFFFFFFFu, dmin, o));
        if (lane == 0 && dmin < (int32_t)kInf16) atomicMin(a.gdiag, dmin);
    }
    // the next step may start its prologue now
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// B0 = P_1 (+ z_row in column-constant mode) in the padded layout, padding
// columns INF; also the caller's slot 0 and g[0] when asked.
__global__ void init_from_dense_kernel(const int16_t *__restrict__ A, int64_t N, int64_t ldb,
                                       const uint16_t *__restrict__ z, uint16_t *__restrict__ B,
                                       int16_t *__restrict__ user0, int32_t *__restrict__ g0) {
    const int64_t q = blockIdx.x;
    int32_t dm = (int32_t)kInf16;
    for (int64_t c = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; c < ldb;
         c += (int64_t)gridDim.y * blockDim.x) {
        uint32_t v = c < N ? (uint32_t)(uint16_t)A[q * N + c] : kInf16;
        B[q * ldb + c] = (uint16_t)(v + (z ? z[q] : 0u));
        if (c < N) {
            if (user0) user0[q * N + c] = (int16_t)v;
            if (c == q) dm = (int32_t)v;
        }
    }
    if (g0 && dm < (int32_t)kInf16) atomicMin(g0, dm);
}

// The same from CSR (transfer matrices are never formed densely here).
// Rows are in the chain's internal order (row q of the CSR is internal row
// q, whose caller row is canon[q]); columns are the caller's, placed at
// colpos[p] in a narrow chain (dropped where it is -1).
__global__ void init_from_csr_kernel(const int64_t *__restrict__ row_ptr,
                                     const int32_t *__restrict__ col, const int16_t *__restrict__ val,
                                     int64_t N, int64_t ldb, const uint16_t *__restrict__ z,
                                     const int32_t *__restrict__ canon,
                                     const int32_t *__restrict__ colpos, uint16_t *__restrict__ B,
                                     int16_t *__restrict__ user0, int32_t *__restrict__ g0,
                                     int64_t col_base) {
    // B holds buffer columns col_base .. col_base + ldb - 1
    const int64_t q = blockIdx.x;
    const int64_t qc = canon ? (int64_t)canon[q] : q;
    const uint16_t zq = z ? z[q] : 0;
    for (int64_t c = threadIdx.x; c < ldb; c += blockDim.x) {
        B[q * ldb + c] = (uint16_t)(kInf16 + zq);
        if (user0 && c < N) user0[qc * N + c] = (int16_t)kInf16;
    }
    __syncthreads();  // the whole row is INF before the arcs land (one block per row)
    for (int64_t e = row_ptr[q] + threadIdx.x; e < row_ptr[q + 1]; e += blockDim.x) {
        const int64_t p = col[e];
        const uint32_t v = (uint32_t)(uint16_t)val[e];
        const int64_t j = (colpos ? (int64_t)colpos[p] : p) - col_base;
        if (j >= 0 && j < ldb) B[q * ldb + j] = (uint16_t)(v + zq);
        if (user0) user0[qc * N + p] = (int16_t)v;
        if (g0 && p == qc) atomicMin(g0, (int32_t)v);
    }
}

// The 8 entries that start at entry R of the 16 held by x and y.
template <int R>
__device__ __forceinline__ uint4 entries_from(const uint4 &x, const uint4 &y) {
    const uint32_t w[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
    uint32_t o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int e = R + 2 * j;
        o[j] = (e & 1) ? __byte_perm(w[e >> 1], w[(e >> 1) + 1], 0x5432) : w[e >> 1];
    }
    return make_uint4(o[0], o[1], o[2], o[3]);
}

// Powers staged in rows of src_ld entries (16-byte aligned) to rows of N
// entries, which start at any 2-byte boundary: per row the entries before
// the first 16-byte boundary of the destination one by one, then aligned
// 16-byte stores, each made of two aligned 16-byte loads of the source
// shifted by the row's offset, then the tail.  One row per block iteration.
__global__ void repack_powers_kernel(const int16_t *__restrict__ src, int64_t src_ld, size_t src_slot,
                                     int16_t *__restrict__ dst, size_t dst_slot, int64_t N, int64_t rows) {
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int64_t k = r / N, i = r - k * N;
        const int16_t *a = src + (size_t)k * src_slot + (size_t)i * (size_t)src_ld;
        int16_t *b = dst + (size_t)k * dst_slot + (size_t)i * (size_t)N;
        const int64_t h0 = (int64_t)(((16 - ((uintptr_t)b & 15)) & 15) >> 1);
        const int head = (int)(h0 < N ? h0 : N);
        const int64_t nb = (N - head) / 8;
        if ((int)threadIdx.x < head) b[threadIdx.x] = a[threadIdx.x];
        for (int64_t t = head + nb * 8 + threadIdx.x; t < N; t += blockDim.x) b[t] = a[t];
        const uint4 *a4 = reinterpret_cast<const uint4 *>(a);
        uint4 *b4 = reinterpret_cast<uint4 *>(b + head);
        // block q of the destination's aligned part takes source entries
        // head + 8q .. head + 8q + 7: the end of source block q and the start
        // of block q + 1 (read only where the shift needs it)
        for (int64_t q = threadIdx.x; q < nb; q += blockDim.x) {
            const uint4 x = a4[q];
            const uint4 y = head ? a4[q + 1] : x;
            uint4 v;
            switch (head) {
                case 0: v = x; break;
                case 1: v = entries_from<1>(x, y); break;
                case 2: v = entries_from<2>(x, y); break;
                case 3: v = entries_from<3>(x, y); break;
                case 4: v = entries_from<4>(x, y); break;
                case 5: v = entries_from<5>(x, y); break;
                case 6: v = entries_from<6>(x, y); break;
                default: v = entries_from<7>(x, y); break;
            }
            b4[q] = v;
        }
    }
}

// Full powers from a narrow chain's chunk-major staging: per pair {i, R i}
// of caller rows the two staged rows gathered into shared memory (16-byte
// pieces, a row's W entries of one chunk contiguous), then both caller rows
// in column order, each entry from one of the two.
__global__ void mirror_repack_kernel(const int16_t *__restrict__ src, int W, int64_t ldb, size_t src_slot,
                                     int16_t *__restrict__ dst, size_t dst_slot, const int32_t *__restrict__ mcol,
                                     const int32_t *__restrict__ mrow, const int32_t *__restrict__ inv,
                                     const int32_t *__restrict__ lead, int64_t nlead, int64_t N, int64_t units,
                                     int *status) {
    extern __shared__ __align__(16) int16_t srow[];  // [2 * ldb]: staged rows of i and of R i
    const int64_t pieces = ldb / 8, ppc = W / 8;     // 16-byte pieces per row, per chunk row
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int64_t k = u / nlead, i = mp_ix((int64_t)lead[u - k * nlead], N, status);
        const int64_t ri = mp_ix((int64_t)mrow[i], N, status);
        const int16_t *base = src + (size_t)k * src_slot;
        const int64_t qa = mp_ix((int64_t)inv[i], N, status), qb = mp_ix((int64_t)inv[ri], N, status);
        __syncthreads();  // the previous pair's reads are done
        for (int64_t t = threadIdx.x; t < 2 * pieces; t += blockDim.x) {
            const int64_t pc = t < pieces ? t : t - pieces, q = t < pieces ? qa : qb;
            const int64_t ch = pc / ppc, h = pc - ch * ppc;
            reinterpret_cast<uint4 *>(srow)[t] =
                *reinterpret_cast<const uint4 *>(base + (size_t)ch * (size_t)N * W + (size_t)q * W + 8 * h);
        }
        __syncthreads();
        int16_t *oa = dst + (size_t)k * dst_slot + (size_t)i * (size_t)N;
        int16_t *ob = dst + (size_t)k * dst_slot + (size_t)ri * (size_t)N;
        for (int64_t c = threadIdx.x; c < N; c += blockDim.x) {
            const int32_t m = mcol[c];
            const int64_t j = mp_ix((int64_t)(m & 0x7FFFFFFF), ldb, status);
            // row i: a kept column from its own row, a mirrored one from row R i;
            // row R i the other way round
            oa[c] = m < 0 ? srow[ldb + j] : srow[j];
            if (ri != i) ob[c] = m < 0 ? srow[j] : srow[ldb + j];
        }
    }
}

// The labelled buffer of a caller's power: internal row q (caller row
// canon[q]), buffer column j (caller column colmap[j], or j), INF beyond the
// kept columns; INF entries stay INF + z like the other initialisations.
__global__ void init_from_power_kernel(const int16_t *__restrict__ P, int64_t N, int64_t ldb,
                                       const uint16_t *__restrict__ z, const int32_t *__restrict__ canon,
                                       const int32_t *__restrict__ colmap, int64_t ncols,
                                       uint16_t *__restrict__ B) {
    const int64_t q = blockIdx.x;
    const int64_t qc = canon ? (int64_t)canon[q] : q;
    const uint32_t zq = z ? z[q] : 0;
    for (int64_t j = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; j < ldb; j += (int64_t)gridDim.y * blockDim.x) {
        uint32_t v = kInf16;
        if (j < ncols) {
            const int64_t c = colmap ? (int64_t)colmap[j] : j;
            v = min((uint32_t)(uint16_t)P[qc * N + c], kInf16);
        }
        B[q * ldb + j] = (uint16_t)(v + zq);
    }
}

// CSR of a dense device matrix (finite = below INF16): warp per row.
__global__ void dense_csr_count_kernel(const int16_t *__restrict__ A, int64_t N,
                                       int64_t *__restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= N) return;
    int64_t c = 0;
    for (int64_t p0 = 0; p0 < N; p0 += 32) {
        int64_t p = p0 + lane;
        bool ok = p < N && (uint16_t)A[q * N + p] < kInf16;
        c += __popc(__ballot_sync(0xFFFFFFFFu, ok));
    }
    if (lane == 0) counts[q] = c;
}

__global__ void dense_csr_fill_kernel(const int16_t *__restrict__ A, int64_t N,
                                      const int64_t *__restrict__ row_ptr, int32_t *__restrict__ col,
                                      int16_t *__restrict__ val) {
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= N) return;
    int64_t pos = row_ptr[q];
    for (int64_t p0 = 0; p0 < N; p0 += 32) {
        int64_t p = p0 + lane;
        int16_t v = p < N ? A[q * N + p] : (int16_t)kInf16;
        bool ok = p < N && (uint16_t)v < kInf16;
        uint32_t bal = __ballot_sync(0xFFFFFFFFu, ok);
        if (ok) {
            int64_t at = pos + __popc(bal & ((1u << lane) - 1u));
            col[at] = (int32_t)p;
            val[at] = v;
        }
        pos += __popc(bal);
    }
}

}  // namespace

// ---------------------------------------------------------------- host side
// (the plan builder, plan_build_host, is in spmm_plan.cu)

int plan_upload(const PlanHost &h, PlanDev *d, cudaStream_t s, bool persistent) {
    d->N = h.N;
    d->ldb = h.ldb;
    d->ngroups = h.ngroups;
    d->nchunks = h.nchunks;
    d->cap_rows = h.cap_rows;
    d->blob_cap = h.blob_cap;
    d->colconst = h.colconst;
    d->nnz = h.nnz;
    auto up = [&](DevBuf &buf, const void *src, size_t bytes) -> int {
        MP_TRY(buf.alloc(bytes ? bytes : 16, s, persistent));
        if (bytes) MP_CUDA_TRY(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, s));
        return MP_OK;
    };
    MP_TRY(up(d->grp_row0, h.grp_row0.data(), h.grp_row0.size() * 4));
    MP_TRY(up(d->grp_stage0, h.grp_stage0.data(), h.grp_stage0.size() * 4));
    MP_TRY(up(d->stage_u0, h.stage_u0.data(), h.stage_u0.size() * 4));
    MP_TRY(up(d->blob_off, h.blob_off.data(), h.blob_off.size() * 8));
    MP_TRY(up(d->blob, h.blob.data(), h.blob.size() * 4));
    // the gathered rows as offsets into the padded power, in 16-byte units
    if (!h.urows.empty() && (double)h.N * (double)h.ldb / 8.0 >= 4294967295.0)
        return set_error(MP_EINVAL, "N = %lld too large for 32-bit row offsets", (long long)h.N);
    std::vector<uint32_t> uoff(h.urows.size());
    for (size_t i = 0; i < uoff.size(); ++i) uoff[i] = (uint32_t)((int64_t)h.urows[i] * (h.ldb / 8));
    MP_TRY(up(d->uoff16, uoff.data(), uoff.size() * 4));
    MP_TRY(up(d->z, h.z.data(), h.z.size() * 2));
    MP_TRY(up(d->units, h.units.data(), h.units.size() * sizeof(UnitDesc)));
    MP_TRY(up(d->cta_unit0, h.cta_unit0.data(), h.cta_unit0.size() * 4));
    d->permuted = !h.canon.empty();
    if (d->permuted) {
        if ((int64_t)h.canon.size() != h.N) return set_error(MP_EINVAL, "row order of the wrong length");
        MP_TRY(up(d->canon, h.canon.data(), h.canon.size() * 4));
    }
    d->narrow = !h.colpos.empty();
    if (d->narrow) {
        if ((int64_t)h.colpos.size() != h.N) return set_error(MP_EINVAL, "column map of the wrong length");
        MP_TRY(up(d->colpos, h.colpos.data(), h.colpos.size() * 4));
    }
    d->grid = h.grid;
    d->h2d_bytes = (h.grp_row0.size() + h.grp_stage0.size() + h.stage_u0.size() + h.blob.size() +
                    h.urows.size() + h.cta_unit0.size()) * 4 + h.blob_off.size() * 8 +
                   h.z.size() * 2 + h.units.size() * sizeof(UnitDesc) + h.canon.size() * 4;
    return MP_OK;
}

int sparse_cap_rows(int *cap_rows, int *blob_cap, int *grid) {
    DeviceInfo di;
    MP_TRY(device_info(&di));
    // one CTA per SM; two buffers, each a 16 KiB blob region plus cap_rows
    // gathered row segments of 128 B (at most kStageRowsMax + the padding
    // row), and the 16 KiB of per-row accumulators
    const int blob = 4096;
    const size_t budget = di.smem_optin - 1024 - kAccBytes - 2 * (size_t)blob * 4;
    int cap = (int)(budget / (2 * (size_t)kRowBytes));
    if (cap > kStageRowsMax + 1) cap = kStageRowsMax + 1;
    *cap_rows = cap;
    *blob_cap = blob;
    *grid = di.sms;
    return MP_OK;
}

int sparse_step(const PlanDev &p, const uint16_t *Bin, uint16_t *Bout, int16_t *user_out,
                int32_t *gdiag, cudaStream_t s) {
    if (p.circuit.ready) return circuit_step(p, Bin, Bout, user_out, gdiag, s);
    if (p.gcircuit.ready) return gcircuit_step(p, Bin, Bout, user_out, gdiag, s);
    if (p.narrow && user_out) return set_error(MP_EINVAL, "a narrow chain has no full powers to write");
    DeviceInfo di;
    MP_TRY(device_info(&di));
    int *status = nullptr;
    MP_TRY(device_status_ptr(&status));
    SpStepArgs a;
    memset(&a, 0, sizeof(a));
    a.uoff16 = p.uoff16.as<uint32_t>();
    a.blob = p.blob.as<uint32_t>();
    a.units = p.units.as<UnitDesc>();
    a.cta_unit0 = p.cta_unit0.as<int32_t>();
    a.cap_rows = p.cap_rows;
    a.blob_cap = p.blob_cap;
    a.N = p.N;
    a.ldb = p.ldb;
    a.Bin = Bin;
    a.Bout = Bout;
    a.user_out = user_out;
    a.gdiag = gdiag;
    a.status = status;
    const size_t smem = 2 * ((size_t)p.blob_cap * 4 + (size_t)p.cap_rows * kRowBytes) + kAccBytes;
    const int64_t grid = p.grid;
    if (grid < 1 || p.N < 1) return MP_OK;
    static bool attr_set[2][64] = {};
    const int kind = p.colconst ? 0 : 1;
    if (di.device < 64 && !attr_set[kind][di.device]) {
        if (p.colconst)
            MP_CUDA_TRY(cudaFuncSetAttribute(sparse_step_kernel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)di.smem_optin));
        else
            MP_CUDA_TRY(cudaFuncSetAttribute(sparse_step_kernel<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)di.smem_optin));
        attr_set[kind][di.device] = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (p.colconst)
        MP_CUDA_TRY(cudaLaunchKernelEx(&cfg, sparse_step_kernel<true>, a));
    else
        MP_CUDA_TRY(cudaLaunchKernelEx(&cfg, sparse_step_kernel<false>, a));
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int sparse_init_from_dense(const PlanDev &p, const int16_t *A, uint16_t *B0, int16_t *user0,
                           int32_t *g0, cudaStream_t s) {
    if (p.permuted) return set_error(MP_EINVAL, "dense initialisation of a reordered plan");
    dim3 grid((unsigned)p.N, (unsigned)std::min<int64_t>((p.ldb + 255) / 256, 64));
    init_from_dense_kernel<<<grid, 256, 0, s>>>(A, p.N, p.ldb, plan_labelled(p) ? p.z.as<uint16_t>() : nullptr,
                                                B0, user0, g0);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int sparse_init_from_csr(const PlanDev &p, const int64_t *row_ptr, const int32_t *col,
                         const int16_t *val, uint16_t *B0, int16_t *user0, int32_t *g0,
                         cudaStream_t s) {
    // one block per row so the INF fill precedes the arc scatter within the block
    dim3 grid((unsigned)p.N, 1);
    if (p.narrow && user0) return set_error(MP_EINVAL, "a narrow chain has no full powers to write");
    init_from_csr_kernel<<<grid, 256, 0, s>>>(row_ptr, col, val, p.N, p.ldb,
                                              plan_labelled(p) ? p.z.as<uint16_t>() : nullptr,
                                              p.permuted ? p.canon.as<int32_t>() : nullptr,
                                              p.narrow ? p.colpos.as<int32_t>() : nullptr, B0,
                                              user0, g0, 0);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int sparse_init_block_from_csr(const PlanDev &p, const int64_t *row_ptr, const int32_t *col,
                               const int16_t *val, int64_t col_base, int64_t width, uint16_t *B0,
                               int32_t *g0, cudaStream_t s) {
    if (col_base < 0 || width < 1 || col_base + width > p.ldb)
        return set_error(MP_EINVAL, "column block out of the plan's buffer");
    dim3 grid((unsigned)p.N, 1);
    init_from_csr_kernel<<<grid, 256, 0, s>>>(row_ptr, col, val, p.N, width,
                                              plan_labelled(p) ? p.z.as<uint16_t>() : nullptr,
                                              p.permuted ? p.canon.as<int32_t>() : nullptr,
                                              p.narrow ? p.colpos.as<int32_t>() : nullptr, B0, nullptr, g0,
                                              col_base);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int launch_repack_powers(const int16_t *src, int64_t src_ld, size_t src_slot, int16_t *dst, size_t dst_slot,
                         int64_t N, int count, cudaStream_t s) {
    if (count < 1 || N < 1) return MP_OK;
    if (src_ld < N || src_ld % 8 || ((uintptr_t)src & 15) || ((uintptr_t)dst & 1))
        return set_error(MP_EINVAL, "repack needs 16-byte aligned source rows and a 2-byte aligned destination");
    const int64_t rows = (int64_t)count * N;
    DeviceInfo di;
    MP_TRY(device_info(&di));
    const unsigned grid = (unsigned)std::min<int64_t>(rows, (int64_t)di.sms * 8);
    repack_powers_kernel<<<grid, 128, 0, s>>>(src, src_ld, src_slot, dst, dst_slot, N, rows);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int launch_mirror_repack(const int16_t *src, int W, int64_t ldb, size_t src_slot, int16_t *dst, size_t dst_slot,
                         const int32_t *mcol, const int32_t *mrow, const int32_t *inv, const int32_t *lead,
                         int64_t nlead, int64_t N, int count, cudaStream_t s) {
    if (count < 1 || N < 1 || nlead < 1) return MP_OK;
    const size_t smem = (size_t)ldb * 4;
    if ((W != 8 && W != 16) || ldb % W || ((uintptr_t)src & 15) || smem > 48 * 1024 ||
        src_slot < (size_t)N * (size_t)ldb)
        return set_error(MP_EINVAL, "mirror repack needs aligned chunks of 8 or 16 columns, rows of at most 6144");
    const int64_t units = (int64_t)count * nlead;
    DeviceInfo di;
    MP_TRY(device_info(&di));
    const unsigned grid = (unsigned)std::min<int64_t>(units, (int64_t)di.sms * 8);
    int *status = nullptr;
    MP_TRY(device_status_ptr(&status));
    mirror_repack_kernel<<<grid, 256, smem, s>>>(src, W, ldb, src_slot, dst, dst_slot, mcol, mrow, inv, lead, nlead,
                                                 N, units, status);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int sparse_init_from_power(const PlanDev &p, const int16_t *P, const int32_t *colmap, int64_t ncols,
                           uint16_t *B0, cudaStream_t s) {
    if (p.N < 1) return MP_OK;
    dim3 grid((unsigned)p.N, (unsigned)std::min<int64_t>((p.ldb + 255) / 256, 16));
    init_from_power_kernel<<<grid, 256, 0, s>>>(P, p.N, p.ldb, plan_labelled(p) ? p.z.as<uint16_t>() : nullptr,
                                                p.permuted ? p.canon.as<int32_t>() : nullptr, colmap, ncols,
                                                B0);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int dense_to_csr(const int16_t *A, int64_t N, HostCsr *csr, DevCsr *dcsr, cudaStream_t s) {
    csr->N = N;
    MP_TRY(dcsr->row_ptr.alloc((size_t)(N + 1) * 8, s));
    int64_t *counts = dcsr->row_ptr.as<int64_t>();
    const int64_t blocks = (N * 32 + 255) / 256;
    dense_csr_count_kernel<<<(unsigned)blocks, 256, 0, s>>>(A, N, counts);
    MP_CUDA_TRY(cudaGetLastError());
    std::vector<int64_t> cnt((size_t)N);
    MP_CUDA_TRY(cudaMemcpyAsync(cnt.data(), counts, (size_t)N * 8, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    csr->row_ptr.assign((size_t)N + 1, 0);
    for (int64_t q = 0; q < N; ++q) csr->row_ptr[q + 1] = csr->row_ptr[q] + cnt[q];
    const int64_t nnz = csr->row_ptr[N];
    MP_CUDA_TRY(cudaMemcpyAsync(counts, csr->row_ptr.data(), (size_t)(N + 1) * 8,
                                cudaMemcpyHostToDevice, s));
    MP_TRY(dcsr->col.alloc((size_t)std::max<int64_t>(nnz, 1) * 4, s));
    MP_TRY(dcsr->val.alloc((size_t)std::max<int64_t>(nnz, 1) * 2, s));
    dense_csr_fill_kernel<<<(unsigned)blocks, 256, 0, s>>>(A, N, counts, dcsr->col.as<int32_t>(),
                                                         dcsr->val.as<int16_t>());
    MP_CUDA_TRY(cudaGetLastError());
    csr->col.resize((size_t)nnz);
    csr->val.resize((size_t)nnz);
    if (nnz) {
        MP_CUDA_TRY(cudaMemcpyAsync(csr->col.data(), dcsr->col.p, (size_t)nnz * 4,
                                    cudaMemcpyDeviceToHost, s));
        MP_CUDA_TRY(cudaMemcpyAsync(csr->val.data(), dcsr->val.p, (size_t)nnz * 2,
                                    cudaMemcpyDeviceToHost, s));
    }
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    return MP_OK;
}

}  // namespace mp
