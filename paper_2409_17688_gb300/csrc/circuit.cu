// K2 by a reuse circuit: the sparse transfer step for column-constant A.
//
// One step of the power chain (Algorithm 2) is P_{k+1} = A (x) P_k.  For the
// transfer matrix every arc into p carries the same label z_p (Section 2.2),
// so with X[p] = z_p + P_k[p] (the chain's labelled buffer) row q of the
// product is R[q] = min over Out(q) of X[p], Out(q) = {p : q -> p}.  Minimum
// is idempotent, so whenever Out(q') is a subset of Out(q) the row R[q'] is a
// partial result of R[q]: R[q] = min(R[q'_1], ..., R[q'_t], min over L(q) of
// X[p]) for any subsets Out(q'_i) whose union with L(q) is Out(q).  The
// words' arc rule makes such subsets plentiful (a letter 2 forces a 0 below
// it, so turning a 1 into a 2 shrinks the successor set), and a greedy cover
// reads at n = 9 about 6.9 rows per output row instead of the 88 arcs of a
// row: 23923 row reads per column against nnz(A) = 303097.  The result is
// the same minimum, bit for bit.
//
// Host: successor sets as bitsets; for each row, in order of set size, the
// rows whose sets it contains, then the greedy cover: take the candidate
// whose coverage of what is still uncovered, less kCircLambda for every
// level it would add to the row, is largest, while that score is at least
// two.  A row's level is one more than the deepest row of its cover; the
// level penalty trades a few more reads for fewer, fuller levels.  Each
// level's rows become lane tasks of at most 8 list entries (one 16-byte
// piece of each row per load): a longer list takes an aligned group of 2,
// 4, .. 32 lanes.  Rows are packed widest first into warp slices of 32
// lanes, so every lane of a level does the same work.
//
// Device (circuit_step_kernel): one CTA per chunk of 8 columns (16 where a
// chain has more 8-column chunks than the GPU has SMs: one CTA per SM then
// spreads the columns evenly).  The circuit (one blob, the same for every
// chunk and every step) is copied into shared memory while the previous
// step finishes, or read from L2 where only the image fits; then the chunk
// of X (N rows of 8 or 16 columns).  The levels run in order with a block
// barrier between them, touching only shared memory: a warp takes every
// 16th slice of a level, each lane folds its 8 rows (the chunk's 16 or 32
// bytes of each), the lanes of a row combine by shuffles and the first of
// them writes the row's result to shared memory for the later levels (a
// single step also writes it, labelled, to the next buffer; a chain adds
// the labels in place after the last level, and the result becomes the next
// step's X).  After the levels the (at most 8 or 16) rows whose diagonal
// entries lie in the chunk are read back and min-reduced into g[k].
#include <algorithm>
#include <cstring>
#include <mutex>

#include "mp_internal.cuh"
#include "spmm.cuh"

namespace mp {

namespace {

constexpr int kCircThreads = 512;
constexpr int kCircWarps = kCircThreads / 32;

__device__ __forceinline__ uint32_t csmem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ccp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ uint32_t clds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint4 clds_v4(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr));
    return v;
}
__device__ __forceinline__ void cmbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void cmbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool cmbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase of the given parity for at most about a second; false
// when the wait ran out.
__device__ __forceinline__ bool cmbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (cmbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!cmbar_try_wait(bar, parity))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}
// bytes (a multiple of 16) from src to dst (both 16-byte aligned), counted on bar.
__device__ __forceinline__ void cbulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void csts_v4(uint32_t addr, uint4 v) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

struct CircArgs {
    const uint16_t *Bin;  // X: the labelled buffer of P_k (P_1 for a chain)
    uint16_t *Bout;       // one step: the labelled buffer of P_{k+1}
    int64_t N, Nh, ldb;
    const uint8_t *meta;
    uint32_t meta_bytes, off_info, off_ents, off_z;
    int levels;
    int k_max;            // a chain: P_2 .. P_{k_max}
    int out_k0;           // a chain: P_k goes to output slot k - out_k0
    int16_t *user_out;    // the caller's power(s), or null
    size_t slot;          // a chain: entries between the caller's powers
    int64_t user_ld;      // entries between rows of a power in user_out: N, or a
                          // multiple of 8 no smaller than ldb (then every piece is
                          // one aligned store, columns past N into the row's padding)
    int chunk_major;      // a chain: user_out takes each power chunk by chunk, the
                          // chunk's rows in the internal order, W entries each,
                          // written by the label pass (consecutive rows: coalesced)
    const int32_t *caller;   // per internal row, the caller's row (for user_out)
    const uint16_t *drow;    // per buffer column, the row whose diagonal entry it holds
    int32_t *gdiag;       // one step: g[k]; a chain: g[0 .. k_max - 1]
    int *status;
    uint32_t extra_tx;    // bytes expected beyond the circuit's (0; > 0 only to inject a timeout)
};

// Byte offset of 16-byte piece h of image row j.  With 8-column chunks a row
// is one piece, in bank group j mod 8.  With 16-column chunks a row is two
// pieces, swapped in rows with bit 2 set, so that piece h of rows with
// distinct j mod 8 still lies in distinct bank groups (2j + (h ^ bit 2 of j)
// mod 8): the entry colouring by j mod 8 holds for both.
template <int kW>
__device__ __forceinline__ uint32_t img_off(uint32_t j, uint32_t h) {
    if (kW == 8) return j * 16u;
    return j * 32u + 16u * (h ^ ((j >> 2) & 1u));
}

// acc = min(acc, the image rows an entry block names), 16 bytes per lane and
// piece; entries naming the INF row (the padding of short lists, index 2Nh)
// load nothing, the others live at image row (index + sh) mod 2Nh.
template <int kW>
__device__ __forceinline__ void fold8(uint4 (&acc)[kW / 8], const uint4 &e, uint32_t rbase, uint32_t N2,
                                      uint32_t sh, int *status) {
    const uint32_t ix[8] = {e.x & 0xFFFFu, e.x >> 16, e.y & 0xFFFFu, e.y >> 16,
                            e.z & 0xFFFFu, e.z >> 16, e.w & 0xFFFFu, e.w >> 16};
    uint32_t jj[8];
#pragma unroll
    for (int h = 0; h < kW / 8; ++h) {
        uint4 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (h == 0) {
                uint32_t j = ix[k] + sh;
                if (j >= N2) j -= N2;
                jj[k] = ix[k] != N2 ? mp_ix(j, N2, status) : 0u;
            }
            v[k] = ix[k] != N2 ? clds_v4(rbase + img_off<kW>(jj[k], (uint32_t)h)) : make_uint4(~0u, ~0u, ~0u, ~0u);
        }
        uint4 &c = acc[h];
        c.x = __vimin3_u16x2(__vimin3_u16x2(c.x, v[0].x, v[1].x), __vimin3_u16x2(v[2].x, v[3].x, v[4].x),
                             __vimin3_u16x2(v[5].x, v[6].x, v[7].x));
        c.y = __vimin3_u16x2(__vimin3_u16x2(c.y, v[0].y, v[1].y), __vimin3_u16x2(v[2].y, v[3].y, v[4].y),
                             __vimin3_u16x2(v[5].y, v[6].y, v[7].y));
        c.z = __vimin3_u16x2(__vimin3_u16x2(c.z, v[0].z, v[1].z), __vimin3_u16x2(v[2].z, v[3].z, v[4].z),
                             __vimin3_u16x2(v[5].z, v[6].z, v[7].z));
        c.w = __vimin3_u16x2(__vimin3_u16x2(c.w, v[0].w, v[1].w), __vimin3_u16x2(v[2].w, v[3].w, v[4].w),
                             __vimin3_u16x2(v[5].w, v[6].w, v[7].w));
    }
}

// Shared memory of a step: the image (X, result, INF row), then the circuit,
// then its copies' mbarrier.
__host__ __device__ __forceinline__ size_t circuit_image_bytes(int64_t N, int W) {
    return ((size_t)(2 * N + 1) * (size_t)(2 * W) + 15) & ~(size_t)15;
}
constexpr uint32_t kCircBarBytes = 16;
constexpr uint32_t kMetaCopy = 32768;  // bytes per bulk copy of the circuit

// One step (kChain false): X from Bin, the result (labelled) to Bout.  A
// chain (kChain true): the CTA runs every step of the chain on its chunk
// without leaving the SM -- column chunk c of P_{k+1} depends only on chunk c
// of P_k -- so after a step the result region, with the labels added in
// place, is the next step's X, and the two regions swap: with sh = 0 or Nh,
// image index j (X rows 0..N-1, result rows Nh..Nh+N-1, Nh = N rounded up to
// 8) lives at (j + sh) mod 2Nh.
// kGBlob: the circuit stays in global memory (read through L1/L2, the next
// slice's lane info and entry block loaded one slice ahead) and only the
// image takes shared memory: chosen where the grid is larger than the GPU's
// SMs, so that two 8-column CTAs fit on an SM (one CTA's barrier waits then
// overlap the other's work) or a 16-column image fits at all.  Otherwise the
// circuit is copied into shared memory.
// The work of one CTA: column chunk bx of the chain (or step) a.
// kW: columns per chunk, 8 (one 16-byte piece per image row) or 16 (two).
// kOut: the code that writes powers (to the caller or a staging area) is
// compiled in (the multi-chain kernel writes none).
template <bool kChain, bool kGBlob, int kW, bool kOut = true>
__device__ __forceinline__ void circuit_body(const CircArgs &a, int bx) {
    constexpr int RB = 2 * kW;  // bytes per image row
    constexpr int NP = kW / 8;  // 16-byte pieces per image row
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t sbase = csmem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t N = a.N;
    const uint32_t Nh = (uint32_t)a.Nh, N2 = 2 * Nh;
    const int64_t c0 = (int64_t)bx * kW;
    const uint32_t mb = sbase + (uint32_t)circuit_image_bytes(Nh, kW);

    // The circuit: plan data only, so its bulk copies start before the
    // previous step has finished.  The barrier's initialisation is made
    // visible to the other threads by the block barrier below, before any of
    // them waits on it.
    const uint32_t copied = kGBlob ? 0u : a.meta_bytes;
    const uint32_t bar = mb + copied;
    if (kGBlob && threadIdx.x == 0) {
        // the circuit is read from L2 at every slice: each CTA brings its share
        // of it into L2 now (plan data, so before the previous kernel ends), so
        // that even the first step after an L2 flush finds it there
        const uint32_t part = 4096u, o = ((uint32_t)bx * part) % ((a.meta_bytes + part - 1) / part * part);
        if (o < a.meta_bytes)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.meta + o),
                         "r"(min(part, a.meta_bytes - o))
                         : "memory");
    }
    if (threadIdx.x == 0) {
        cmbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        cmbar_arrive_expect_tx(bar, copied + a.extra_tx);
        if (!kGBlob)
            for (uint32_t o = 0; o < a.meta_bytes; o += kMetaCopy)
                cbulk_copy(mb + o, a.meta + o, min(kMetaCopy, a.meta_bytes - o), bar);
    }
    // row 2Nh of the image: above every value, the padding of short lists
    if (threadIdx.x < RB / 4) reinterpret_cast<uint32_t *>(smem + (size_t)N2 * RB)[threadIdx.x] = 0xFFFFFFFFu;
    // the row whose diagonal entry lies in column c0 + t (threads t < kW)
    uint32_t drow = 0xFFFFu;
    if (a.gdiag && threadIdx.x < kW) drow = a.drow[mp_ix(c0 + (int64_t)threadIdx.x, a.ldb, a.status)];
    // Programmatic dependent launch: the previous step's output (our X) is
    // read only after its grid has completed.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // X's chunk: N rows of RB bytes
    for (int64_t r = threadIdx.x; r < N; r += kCircThreads)
#pragma unroll
        for (int h = 0; h < NP; ++h)
            ccp_async16(sbase + img_off<kW>((uint32_t)r, (uint32_t)h),
                        a.Bin + r * a.ldb + mp_ix(c0 + 8 * h, a.ldb - 7, a.status));
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // the circuit's copies; a wait that ran out stops the whole block (after
    // a second bounded wait, so no copy lands after it has gone)
    const bool landed = cmbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!landed)) {
        if (threadIdx.x == 0) atomicCAS(a.status, 0, MP_ETIMEOUT);
        cmbar_wait_bounded(bar, 0);
        return;
    }

    const uint32_t m_info = mb + a.off_info, m_en = mb + a.off_ents, m_z = mb + a.off_z;
    const uint32_t *g_lvl = reinterpret_cast<const uint32_t *>(a.meta);
    const uint32_t *g_info = reinterpret_cast<const uint32_t *>(a.meta + a.off_info);
    const uint4 *g_ents = reinterpret_cast<const uint4 *>(a.meta + a.off_ents);
    const uint16_t *g_z = reinterpret_cast<const uint16_t *>(a.meta + a.off_z);
    auto label = [&](uint32_t q) {
        q = mp_ix(q, (uint32_t)N, a.status);
        if (kGBlob) return (uint32_t)__ldg(g_z + q);
        const uint32_t zw = clds_u32(m_z + 4u * (q >> 1));
        return (q & 1) ? zw >> 16 : zw & 0xFFFFu;
    };
    auto level_start = [&](int l) { return kGBlob ? (int)__ldg(g_lvl + l) : (int)clds_u32(mb + 4u * (uint32_t)l); };
    const int nsl = level_start(a.levels);  // warp slices of the circuit
    auto slice_info = [&](int sl) {
        sl = mp_ix(sl, nsl, a.status);
        return kGBlob ? __ldg(g_info + (size_t)sl * 32 + lane) : clds_u32(m_info + 4u * ((uint32_t)sl * 32u + (uint32_t)lane));
    };
    auto slice_ents = [&](int sl) {
        sl = mp_ix(sl, nsl, a.status);
        return kGBlob ? __ldg(g_ents + (size_t)sl * 32 + lane) : clds_v4(m_en + 16u * ((uint32_t)sl * 32u + (uint32_t)lane));
    };
    // the label of the row whose diagonal entry lies in this thread's column
    const uint32_t zdrow = (kChain && drow != 0xFFFFu) ? label(drow) : 0u;
    const int k_last = kChain ? a.k_max : 2;
    uint32_t sh = 0;
    // From global memory a slice's lane info and entry block are read one
    // slice ahead, and the first slice of the next level (of the next step's
    // first level after the last) before the barrier that ends a level: the
    // circuit is plan data, so nothing orders these reads after the barrier.
    uint32_t info_n = 0;
    uint4 e_n = make_uint4(0, 0, 0, 0);
    if (kGBlob && level_start(0) + warp < level_start(1)) {
        info_n = slice_info(level_start(0) + warp);
        e_n = slice_ents(level_start(0) + warp);
    }
    for (int k = 2; k <= k_last; ++k) {
        for (int l = 0; l < a.levels; ++l) {
            const int s1 = level_start(l + 1);
            int s = level_start(l) + warp;
            for (; s < s1; s += kCircWarps) {
                uint32_t info;
                uint4 e_c;
                if (kGBlob) {
                    info = info_n;
                    e_c = e_n;
                    if (s + kCircWarps < s1) {
                        info_n = slice_info(s + kCircWarps);
                        e_n = slice_ents(s + kCircWarps);
                    }
                } else {
                    info = slice_info(s);
                    e_c = slice_ents(s);
                }
                uint4 acc[NP];
#pragma unroll
                for (int h = 0; h < NP; ++h) acc[h] = make_uint4(kInf16x2, kInf16x2, kInf16x2, kInf16x2);
                fold8<kW>(acc, e_c, sbase, N2, sh, a.status);
                // the lanes of one row (an aligned group of 1 << lg) combine;
                // the slice's widest row sits in lane 0
                const uint32_t lg = (info >> 16) & 7u;
                const uint32_t lg0 = __shfl_sync(0xFFFFFFFFu, lg, 0);
                for (uint32_t o = 1; o < (1u << lg0); o <<= 1) {
#pragma unroll
                    for (int h = 0; h < NP; ++h) {
                        const uint32_t vx = __shfl_xor_sync(0xFFFFFFFFu, acc[h].x, o);
                        const uint32_t vy = __shfl_xor_sync(0xFFFFFFFFu, acc[h].y, o);
                        const uint32_t vz = __shfl_xor_sync(0xFFFFFFFFu, acc[h].z, o);
                        const uint32_t vw = __shfl_xor_sync(0xFFFFFFFFu, acc[h].w, o);
                        if (o < (1u << lg))
                            acc[h] = make_uint4(__vminu2(acc[h].x, vx), __vminu2(acc[h].y, vy),
                                                __vminu2(acc[h].z, vz), __vminu2(acc[h].w, vw));
                    }
                }
                const uint32_t q = info & 0xFFFFu;
                if (q == 0xFFFFu || (lane & ((1u << lg) - 1u)) != 0) continue;
                // the result row, for the later levels (and the next step)
                uint32_t rr = Nh + q + sh;
                if (rr >= N2) rr -= N2;
                rr = mp_ix(rr, N2, a.status);
#pragma unroll
                for (int h = 0; h < NP; ++h) csts_v4(sbase + img_off<kW>(rr, (uint32_t)h), acc[h]);
                if (!kChain) {
                    const uint32_t zq = label(q) * 0x10001u;
#pragma unroll
                    for (int h = 0; h < NP; ++h)
                        *reinterpret_cast<uint4 *>(a.Bout + (int64_t)q * a.ldb + c0 + 8 * h) =
                            make_uint4(acc[h].x + zq, acc[h].y + zq, acc[h].z + zq, acc[h].w + zq);
                }
                if (kOut && a.user_out && !(kChain && a.chunk_major)) {
                    int16_t *dst = a.user_out + (kChain ? (size_t)(k - a.out_k0) * a.slot : 0) +
                                   (int64_t)mp_ix((int64_t)a.caller[q], N, a.status) * a.user_ld + c0;
#pragma unroll
                    for (int h = 0; h < NP; ++h) {
                        if (a.user_ld % 8 == 0 && a.user_ld >= a.ldb)
                            *reinterpret_cast<uint4 *>(dst + 8 * h) = acc[h];
                        else
                            store_row8(dst + 8 * h, acc[h], N - c0 - 8 * h);
                    }
                }
            }
            if (kGBlob) {
                const int nl = l + 1 < a.levels ? l + 1 : 0;
                const int ns = level_start(nl) + warp;
                if (ns < level_start(nl + 1)) {
                    info_n = slice_info(ns);
                    e_n = slice_ents(ns);
                }
            }
            __syncthreads();  // this level's rows are read by the later levels
        }
        const uint32_t shr = sh;  // where this step's result rows are
        if (kChain) {
            // the labels, in place: the result becomes the next step's X (the
            // labels of four rows per thread loaded before their rows); a
            // chain staging its powers chunk by chunk writes each row first
            int16_t *stage = (kOut && a.user_out && a.chunk_major)
                                 ? a.user_out + (size_t)(k - a.out_k0) * a.slot + (size_t)bx * (size_t)N * kW
                                 : nullptr;
            for (uint32_t q0 = threadIdx.x; q0 < (uint32_t)N; q0 += 4 * kCircThreads) {
                uint32_t zq[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t q = q0 + (uint32_t)j * kCircThreads;
                    zq[j] = q < (uint32_t)N ? label(q) * 0x10001u : 0u;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t q = q0 + (uint32_t)j * kCircThreads;
                    if (q >= (uint32_t)N) break;
                    uint32_t rr = Nh + q + sh;
                    if (rr >= N2) rr -= N2;
                    rr = mp_ix(rr, N2, a.status);
#pragma unroll
                    for (int h = 0; h < NP; ++h) {
                        const uint32_t addr = sbase + img_off<kW>(rr, (uint32_t)h);
                        const uint4 v = clds_v4(addr);
                        if (stage) *reinterpret_cast<uint4 *>(stage + (size_t)q * kW + 8 * h) = v;
                        csts_v4(addr, make_uint4(v.x + zq[j], v.y + zq[j], v.z + zq[j], v.w + zq[j]));
                    }
                }
            }
            sh = Nh - sh;
            __syncthreads();
        }
        if (a.gdiag && warp == 0) {
            // the diagonal entries of this chunk (unlabelled); the next step
            // writes only the other region, so nothing races with these reads
            int32_t v = (int32_t)kInf16;
            if (lane < kW && drow != 0xFFFFu) {
                uint32_t rr = Nh + drow + shr;
                if (rr >= N2) rr -= N2;
                rr = mp_ix(rr, N2, a.status);
                const uint32_t w =
                    clds_u32(sbase + img_off<kW>(rr, (uint32_t)lane >> 3) + 4u * (uint32_t)((lane & 7) >> 1));
                v = (int32_t)((lane & 1) ? w >> 16 : w & 0xFFFFu);
                if (kChain) v -= (int32_t)zdrow;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
            if (lane == 0 && v < (int32_t)kInf16) atomicMin(kChain ? a.gdiag + (k - a.out_k0) : a.gdiag, v);
        }
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <bool kChain, bool kGBlob, int kW>
__global__ void __launch_bounds__(kCircThreads, kGBlob && kW == 8 ? 2 : 1) circuit_step_kernel(CircArgs a) {
    circuit_body<kChain, kGBlob, kW>(a, (int)blockIdx.x);
}

// Several chains in one launch: the CTAs of chain i are blocks
// cta0[i] .. cta0[i + 1] - 1, the chains in the order given (longest first),
// so the longest chain's CTAs are placed on the SMs first and the short
// chains fill what is left, whatever the timing of the launches.  A CTA of
// chain i runs its chunks b, b + ctas_i, ... one after another (chunks[i] in
// all), so that the short chains fit into the waves the longest needs.
constexpr int kMultiChains = 8;
struct MultiCircArgs {
    CircArgs c[kMultiChains];
    int cta0[kMultiChains + 1];
    int chunks[kMultiChains];
    int count;
};

template <bool kGBlob, int kW>
__global__ void __launch_bounds__(kCircThreads, kGBlob && kW == 8 ? 2 : 1)
    circuit_multi_kernel(const __grid_constant__ MultiCircArgs m) {
    int ci = 0;
    while (ci + 1 < m.count && (int)blockIdx.x >= m.cta0[ci + 1]) ++ci;
    const int ctas = m.cta0[ci + 1] - m.cta0[ci];
    // this chain's arguments in registers: read through the chain index, every
    // use in the step loops would be a load from the parameter space
    const CircArgs a = m.c[ci];
    for (int bx = (int)blockIdx.x - m.cta0[ci]; bx < m.chunks[ci]; bx += ctas) {
        circuit_body<true, kGBlob, kW, false>(a, bx);
        __syncthreads();  // shared memory and the mbarrier are set up again for the next chunk
    }
}

}  // namespace

int circuit_cover_host(const HostCsr &csr, CircuitCover *out, int lambda) {
    const int64_t N = csr.N;
    if (N < 1 || 2 * N + 1 > 0xFFFF) return set_error(MP_EINVAL, "N = %lld too large for a circuit", (long long)N);
    if (lambda < 0) return set_error(MP_EINVAL, "level penalty %d < 0", lambda);
    CircuitCover &C = *out;
    C = CircuitCover();
    C.N = N;
    const int64_t nw = (N + 63) / 64;
    std::vector<uint64_t> S((size_t)(N * nw), 0);
    std::vector<int64_t> sz((size_t)N);
    for (int64_t q = 0; q < N; ++q) {
        for (int64_t e = csr.row_ptr[q]; e < csr.row_ptr[q + 1]; ++e) {
            const int64_t p = csr.col[e];
            if (p < 0 || p >= N) return set_error(MP_EINVAL, "column %lld out of range", (long long)p);
            uint64_t &wd = S[(size_t)(q * nw + p / 64)];
            if (wd >> (p % 64) & 1) return set_error(MP_EINVAL, "row %lld repeats an arc", (long long)q);
            wd |= 1ull << (p % 64);
        }
        sz[(size_t)q] = csr.row_ptr[q + 1] - csr.row_ptr[q];
    }
    // rows by set size (then index): every cover row precedes its row
    std::vector<int64_t> order((size_t)N);
    for (int64_t q = 0; q < N; ++q) order[(size_t)q] = q;
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t x, int64_t y) { return sz[(size_t)x] < sz[(size_t)y]; });
    C.lists.assign((size_t)N, {});
    C.level.assign((size_t)N, 0);
    std::vector<uint64_t> U((size_t)nw);
    std::vector<int64_t> cand;
    for (int64_t t = 0; t < N; ++t) {
        const int64_t q = order[(size_t)t];
        const uint64_t *Sq = &S[(size_t)(q * nw)];
        cand.clear();
        for (int64_t u = 0; u < t; ++u) {
            const int64_t c = order[(size_t)u];
            if (sz[(size_t)c] < 2) continue;  // covering a single arc saves nothing
            const uint64_t *Sc = &S[(size_t)(c * nw)];
            bool in = true;
            for (int64_t w = 0; w < nw && in; ++w) in = (Sc[w] & ~Sq[w]) == 0;
            if (in) cand.push_back(c);
        }
        std::copy(Sq, Sq + nw, U.begin());
        std::vector<uint32_t> &li = C.lists[(size_t)q];
        int lv = 0;
        while (!cand.empty()) {
            // score: arcs still uncovered that the candidate covers, less the
            // penalty for each level it adds to this row; a cover must score
            // at least two (one read for two or more)
            int64_t best = -1, bs = 1;
            size_t bi = 0;
            for (size_t k = 0; k < cand.size(); ++k) {
                const uint64_t *Sc = &S[(size_t)(cand[k] * nw)];
                int64_t g = 0;
                for (int64_t w = 0; w < nw; ++w) g += __builtin_popcountll(Sc[w] & U[(size_t)w]);
                const int64_t added = std::max(0, C.level[(size_t)cand[k]] + 1 - lv);
                const int64_t sc = g - (int64_t)lambda * added;
                if (g > 1 && sc > bs) {
                    bs = sc;
                    best = cand[k];
                    bi = k;
                }
            }
            if (best < 0) break;  // nothing left worth a cover: read the rest directly
            const uint64_t *Sb = &S[(size_t)(best * nw)];
            for (int64_t w = 0; w < nw; ++w) U[(size_t)w] &= ~Sb[w];
            li.push_back((uint32_t)(N + best));
            lv = std::max(lv, C.level[(size_t)best] + 1);
            cand.erase(cand.begin() + (long)bi);
            ++C.cover_reads;
        }
        for (int64_t w = 0; w < nw; ++w)
            for (uint64_t b = U[(size_t)w]; b; b &= b - 1)
                li.push_back((uint32_t)(w * 64 + __builtin_ctzll(b)));
        C.level[(size_t)q] = lv;
        C.reads += (int64_t)li.size();
        C.levels = std::max(C.levels, lv + 1);
    }
    return MP_OK;
}

int circuit_slice_host(const CircuitCover &cv, CircuitHost *out) {
    const int64_t N = cv.N;
    CircuitHost &C = *out;
    C = CircuitHost();
    C.N = N;
    C.Nh = (N + 7) & ~(int64_t)7;
    C.W = kCircW;
    C.levels = cv.levels;
    C.reads = cv.reads;
    C.cover_reads = cv.cover_reads;
    if (2 * C.Nh + 1 > 0xFFFF || N >= 0xFFFF)
        return set_error(MP_EINVAL, "N = %lld too large for a circuit", (long long)N);
    const uint16_t pad = (uint16_t)(2 * C.Nh);
    // a list entry in image rows: X rows stay, result row N + q' moves to Nh + q'
    auto img = [&](uint32_t v) { return v < (uint32_t)N ? v : v - (uint32_t)N + (uint32_t)C.Nh; };
    auto lanes_log2 = [](size_t len) {
        int lg = 0;
        while (((size_t)8 << lg) < len) ++lg;
        return lg;
    };
    C.level_slice0.push_back(0);
    for (int l = 0; l < C.levels; ++l) {
        // this level's rows, widest first
        std::vector<std::vector<int64_t>> by_lg(6);
        for (int64_t q = 0; q < N; ++q) {
            if (cv.level[(size_t)q] != l) continue;
            const int lg = lanes_log2(cv.lists[(size_t)q].size());
            if ((1 << lg) > kCircLaneMax)
                return set_error(MP_EINVAL, "row %lld reads %zu rows: too many for one warp", (long long)q,
                                 cv.lists[(size_t)q].size());
            by_lg[(size_t)lg].push_back(q);
        }
        std::vector<int64_t> seq;
        for (int lg = 5; lg >= 1; --lg) seq.insert(seq.end(), by_lg[(size_t)lg].begin(), by_lg[(size_t)lg].end());
        {
            // One-lane rows, longest list first, grouped eight at a time into
            // quarter warps.  Under the colouring below a quarter takes about
            // max(longest list, fullest bank group) passes per block, so a
            // quarter starts with the longest row left and takes, from the
            // next rows in that order, the one that keeps its fullest bank
            // group smallest.  The quarters line up with the hardware's only
            // after the multi-lane rows, which fill whole groups of lanes.
            std::vector<int64_t> rows1 = by_lg[0];
            std::stable_sort(rows1.begin(), rows1.end(), [&](int64_t x, int64_t y) {
                return cv.lists[(size_t)x].size() > cv.lists[(size_t)y].size();
            });
            auto hist = [&](int64_t q, int *h) {
                for (uint32_t v : cv.lists[(size_t)q]) ++h[img(v) % 8];
            };
            size_t lane_at = 0;
            for (int64_t q : seq) lane_at += (size_t)1 << lanes_log2(cv.lists[(size_t)q].size());
            std::vector<char> taken(rows1.size(), 0);
            size_t first = 0;  // first row not yet taken
            const size_t window = 48;
            int H[8] = {0};
            while (first < rows1.size()) {
                if (lane_at % 8 == 0) std::fill(H, H + 8, 0);
                size_t best = rows1.size();
                int best_max = 1 << 30, best_sq = 1 << 30;
                for (size_t t = first, seen = 0; t < rows1.size() && seen < window; ++t) {
                    if (taken[t]) continue;
                    ++seen;
                    int h[8];
                    std::copy(H, H + 8, h);
                    hist(rows1[t], h);
                    int mx = 0, sq = 0;
                    for (int r = 0; r < 8; ++r) {
                        mx = std::max(mx, h[r]);
                        sq += h[r] * h[r];
                    }
                    // the quarter's first row is the longest left
                    if (lane_at % 8 == 0) {
                        best = t;
                        break;
                    }
                    if (mx < best_max || (mx == best_max && sq < best_sq)) {
                        best = t;
                        best_max = mx;
                        best_sq = sq;
                    }
                }
                taken[best] = 1;
                hist(rows1[best], H);
                seq.push_back(rows1[best]);
                ++lane_at;
                while (first < rows1.size() && taken[first]) ++first;
            }
        }
        // lanes: row q takes an aligned group of 1 << lg lanes (widest first,
        // so every group starts at a multiple of its size)
        std::vector<int64_t> lane_row;  // -1: idle
        for (int64_t q : seq) {
            const int g = 1 << lanes_log2(cv.lists[(size_t)q].size());
            for (int i = 0; i < g; ++i) lane_row.push_back(q);
        }
        while (lane_row.size() % 32) lane_row.push_back(-1);
        const size_t nsl = lane_row.size() / 32;
        for (size_t sl = 0; sl < nsl; ++sl) {
            const int64_t *lr = &lane_row[sl * 32];
            // Each row's list spread over its lanes and over the 8 positions
            // of the lanes' blocks (min is order-free), chosen so that at every
            // position the loads spread over the shared-memory banks: an image
            // row of 16 bytes sits in bank group (row mod 8) and a 16-byte load
            // is served a quarter warp (8 lanes) at a time, taking as many
            // passes as its fullest group.  A row's entries are dealt to its
            // lanes by group; then per quarter the entries are the edges of a
            // bipartite multigraph between its 8 lanes and the 8 groups, and
            // positions are colours: a proper edge colouring (alternating-path
            // construction; a bipartite graph of largest degree D needs only D
            // colours) makes every position conflict-free.  Where a group holds
            // more than 8 of the quarter's entries, the edges coloured 8 and
            // above go to a position free at their lane whose group count is
            // lowest.  The result rows start at a multiple of 8, so the
            // regions' swap in a chain keeps every row's group.
            std::vector<std::vector<uint32_t>> rem(32);
            for (int i = 0; i < 32; ++i) {
                if (lr[i] < 0 || (i > 0 && lr[i - 1] == lr[i])) continue;
                int g = 1;
                while (i + g < 32 && lr[i + g] == lr[i]) ++g;
                std::vector<uint32_t> li;
                for (uint32_t v : cv.lists[(size_t)lr[i]]) li.push_back(img(v));
                std::stable_sort(li.begin(), li.end(), [](uint32_t x, uint32_t y) { return x % 8 < y % 8; });
                for (size_t t = 0; t < li.size(); ++t) rem[(size_t)i + t % (size_t)g].push_back(li[t]);
            }
            std::vector<uint16_t> blk(32 * 8, pad);
            for (int qw = 0; qw < 4; ++qw) {
                // edges: (lane, group) per entry; colour[e] = position
                std::vector<int> eu, ev;
                std::vector<uint32_t> eval;
                for (int i = 0; i < 8; ++i)
                    for (uint32_t v : rem[(size_t)(qw * 8 + i)]) {
                        eu.push_back(i);
                        ev.push_back((int)(v % 8));
                        eval.push_back(v);
                    }
                const int E = (int)eu.size();
                int D = 8;
                {
                    int dv[8] = {0};
                    for (int e = 0; e < E; ++e) D = std::max(D, ++dv[ev[(size_t)e]]);
                }
                // at[u][c] / bt[v][c]: the edge of colour c at lane u / group v
                std::vector<int> at((size_t)8 * D, -1), bt((size_t)8 * D, -1), col((size_t)E, -1);
                for (int e = 0; e < E; ++e) {
                    const int u = eu[(size_t)e], v = ev[(size_t)e];
                    int ca = 0, cb = 0;
                    while (at[(size_t)u * D + ca] >= 0) ++ca;  // free at u
                    while (bt[(size_t)v * D + cb] >= 0) ++cb;  // free at v
                    if (bt[(size_t)v * D + ca] >= 0) {
                        // swap colours ca and cb along the path from v that
                        // alternates ca, cb, ...; it cannot reach u
                        std::vector<int> path;
                        int x = v, side = 1, c = ca;
                        while (true) {
                            const int f = side ? bt[(size_t)x * D + c] : at[(size_t)x * D + c];
                            if (f < 0) break;
                            path.push_back(f);
                            x = side ? eu[(size_t)f] : ev[(size_t)f];
                            side ^= 1;
                            c = c == ca ? cb : ca;
                        }
                        for (int f : path) {
                            at[(size_t)eu[(size_t)f] * D + col[(size_t)f]] = -1;
                            bt[(size_t)ev[(size_t)f] * D + col[(size_t)f]] = -1;
                        }
                        for (int f : path) {
                            col[(size_t)f] = col[(size_t)f] == ca ? cb : ca;
                            at[(size_t)eu[(size_t)f] * D + col[(size_t)f]] = f;
                            bt[(size_t)ev[(size_t)f] * D + col[(size_t)f]] = f;
                        }
                    }
                    col[(size_t)e] = ca;
                    at[(size_t)u * D + ca] = e;
                    bt[(size_t)v * D + ca] = e;
                }
                // positions 0..7 as coloured; overflow edges where their lane
                // is free and their group least used
                int cnt[8][8] = {};
                std::vector<int> over;
                for (int e = 0; e < E; ++e) {
                    if (col[(size_t)e] < 8) {
                        blk[(size_t)(qw * 8 + eu[(size_t)e]) * 8 + (size_t)col[(size_t)e]] = (uint16_t)eval[(size_t)e];
                        ++cnt[col[(size_t)e]][ev[(size_t)e]];
                    } else {
                        over.push_back(e);
                    }
                }
                for (int e : over) {
                    const int u = eu[(size_t)e], v = ev[(size_t)e];
                    int bestp = -1;
                    for (int p8 = 0; p8 < 8; ++p8)
                        if (blk[(size_t)(qw * 8 + u) * 8 + (size_t)p8] == pad &&
                            (bestp < 0 || cnt[p8][v] < cnt[bestp][v]))
                            bestp = p8;
                    if (bestp < 0) return set_error(MP_EINVAL, "circuit lane with more than 8 entries");
                    blk[(size_t)(qw * 8 + u) * 8 + (size_t)bestp] = (uint16_t)eval[(size_t)e];
                    ++cnt[bestp][v];
                }
                for (int i = 0; i < 8; ++i) rem[(size_t)(qw * 8 + i)].clear();
            }
            for (int i = 0; i < 32; ++i) {
                if (lr[i] >= 0 && !rem[(size_t)i].empty())
                    return set_error(MP_EINVAL, "circuit slicing left entries of row %lld", (long long)lr[i]);
                const int lg = lr[i] >= 0 ? lanes_log2(cv.lists[(size_t)lr[i]].size()) : 0;
                C.info.push_back(lr[i] >= 0 ? (uint32_t)lr[i] | ((uint32_t)lg << 16) : 0xFFFFu);
                C.lanes += lr[i] >= 0;
            }
            C.ents.insert(C.ents.end(), blk.begin(), blk.end());
        }
        C.level_slice0.push_back(C.level_slice0.back() + (int32_t)nsl);
    }
    return MP_OK;
}

int circuit_build_host(const HostCsr &csr, CircuitHost *out) {
    CircuitCover cv;
    MP_TRY(circuit_cover_host(csr, &cv));
    return circuit_slice_host(cv, out);
}

// Section offsets of the circuit blob (bytes, each section a multiple of 16).
struct CircLayout {
    uint32_t info = 0, ents = 0, z = 0, total = 0;
};
static CircLayout circuit_layout(const CircuitHost &h) {
    auto r16 = [](size_t b) { return (uint32_t)((b + 15) & ~(size_t)15); };
    CircLayout L;
    L.info = r16(h.level_slice0.size() * 4);
    L.ents = L.info + r16(h.info.size() * 4);
    L.z = L.ents + r16(h.ents.size() * 2);
    L.total = L.z + r16((size_t)h.N * 2);  // the rows' labels
    return L;
}

int circuit_smem_bytes(const CircuitHost &h, size_t *bytes) {
    *bytes = circuit_image_bytes(h.Nh, kCircW) + circuit_layout(h).total + kCircBarBytes;
    DeviceInfo di;
    MP_TRY(device_info(&di));
    if (*bytes + 1024 > di.smem_optin) *bytes = 0;  // a margin for the kernel's static shared memory
    return MP_OK;
}

int circuit_upload(const CircuitHost &h, const std::vector<uint16_t> &z,
                   const std::vector<int32_t> &diagcol, const std::vector<int32_t> &caller,
                   PlanDev *d, cudaStream_t s) {
    CircuitDev &c = d->circuit;
    c.ready = false;
    if ((int64_t)diagcol.size() != h.N || (int64_t)z.size() != h.N || (int64_t)caller.size() != h.N ||
        h.N != d->N || h.W != kCircW)
        return set_error(MP_EINVAL, "circuit of the wrong size");
    if (d->ldb % kCircW) return set_error(MP_EINVAL, "circuit width does not divide the buffer");
    const CircLayout L = circuit_layout(h);
    std::vector<uint8_t> blob(L.total, 0);
    memcpy(blob.data(), h.level_slice0.data(), h.level_slice0.size() * 4);
    memcpy(blob.data() + L.info, h.info.data(), h.info.size() * 4);
    memcpy(blob.data() + L.ents, h.ents.data(), h.ents.size() * 2);
    for (int64_t q = 0; q < h.N; ++q)
        if (z[(size_t)q] > 0x7FFFu) return set_error(MP_EINVAL, "circuit label out of range");
    memcpy(blob.data() + L.z, z.data(), z.size() * 2);
    std::vector<uint16_t> drow((size_t)d->ldb, 0xFFFFu);
    for (int64_t q = 0; q < h.N; ++q) {
        const int32_t dc = diagcol[(size_t)q];
        if (dc >= (int32_t)d->ldb || caller[(size_t)q] < 0)
            return set_error(MP_EINVAL, "circuit row fields out of range");
        if (dc >= 0) drow[(size_t)dc] = (uint16_t)q;
    }
    MP_TRY(c.meta.alloc(L.total ? L.total : 16, s, true));
    MP_TRY(c.drow.alloc(drow.size() * 2, s, true));
    MP_TRY(c.caller.alloc((size_t)h.N * 4, s, true));
    MP_CUDA_TRY(cudaMemcpyAsync(c.meta.p, blob.data(), L.total, cudaMemcpyHostToDevice, s));
    MP_CUDA_TRY(cudaMemcpyAsync(c.drow.p, drow.data(), drow.size() * 2, cudaMemcpyHostToDevice, s));
    MP_CUDA_TRY(cudaMemcpyAsync(c.caller.p, caller.data(), (size_t)h.N * 4, cudaMemcpyHostToDevice, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors go out of scope
    c.W = kCircW;
    c.Nh = h.Nh;
    c.levels = h.levels;
    c.nslices = (int64_t)h.level_slice0.back();
    c.meta_bytes = L.total;
    c.off_info = L.info;
    c.off_ents = L.ents;
    c.off_z = L.z;
    c.ready = true;
    return MP_OK;
}

static int circuit_args(const PlanDev &p, const uint16_t *Bin, uint16_t *Bout, int k_max, int16_t *user_out,
                        size_t slot, int64_t user_ld, int32_t *gdiag, uint32_t extra_tx, int out_k0,
                        CircArgs *out, bool chunk_major = false) {
    const CircuitDev &c = p.circuit;
    if (!c.ready) return set_error(MP_EINVAL, "plan has no circuit");
    if (p.narrow && user_out && (user_ld == 0 || user_ld == p.N))
        return set_error(MP_EINVAL, "a narrow chain writes its powers in buffer columns only");
    CircArgs &a = *out;
    memset(&a, 0, sizeof(a));
    a.Bin = Bin;
    a.Bout = Bout;
    a.N = p.N;
    a.Nh = c.Nh;
    a.ldb = p.ldb;
    a.meta = c.meta.as<uint8_t>();
    a.meta_bytes = c.meta_bytes;
    a.off_info = c.off_info;
    a.off_ents = c.off_ents;
    a.off_z = c.off_z;
    a.levels = c.levels;
    a.k_max = k_max;
    a.out_k0 = out_k0;
    a.user_out = user_out;
    a.slot = slot;
    if (user_ld == 0) user_ld = p.N;
    if (user_out && user_ld != p.N && (user_ld % 8 || user_ld < p.ldb))
        return set_error(MP_EINVAL, "power rows of %lld entries: need N or a multiple of 8 >= %lld",
                         (long long)user_ld, (long long)p.ldb);
    a.user_ld = user_ld;
    a.chunk_major = chunk_major ? 1 : 0;
    if (chunk_major && (!user_out || slot < (size_t)p.N * (size_t)p.ldb))
        return set_error(MP_EINVAL, "chunk-major staging needs N x ldb entries per power");
    a.caller = c.caller.as<int32_t>();
    a.drow = c.drow.as<uint16_t>();
    a.gdiag = gdiag;
    a.extra_tx = extra_tx;
    return device_status_ptr(&a.status);
}

// The dynamic shared memory a kernel may take, raised as larger plans come.
template <class Kern>
static int circuit_attr(Kern kern, int kind, bool gblob, size_t smem, const DeviceInfo &di) {
    static std::mutex attr_mu;
    static size_t attr_set[8][64] = {};
    std::lock_guard<std::mutex> lk(attr_mu);
    if (di.device >= 64 || attr_set[kind][di.device] < smem) {
        MP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (gblob)
            MP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared));
        if (di.device < 64) attr_set[kind][di.device] = smem;
    }
    return MP_OK;
}

template <class Kern, class Args>
static int circuit_kick(Kern kern, const Args &a, unsigned grid, size_t smem, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kCircThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MP_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

// One launch: a step (Bin -> Bout) or a whole chain from Bin = P_1.
static int circuit_launch(const PlanDev &p, bool chain, const uint16_t *Bin, uint16_t *Bout, int k_max,
                          int16_t *user_out, size_t slot, int32_t *gdiag, cudaStream_t s,
                          uint32_t extra_tx = 0, int out_k0 = 1, int64_t user_ld = 0, int *width = nullptr) {
    DeviceInfo di;
    MP_TRY(device_info(&di));
    CircArgs a;
    const bool chunk_major = width != nullptr;
    MP_TRY(circuit_args(p, Bin, Bout, k_max, user_out, slot, user_ld, gdiag, extra_tx, out_k0, &a, chunk_major));
    if (chunk_major && !chain) return set_error(MP_EINVAL, "chunk-major staging is for chains");
    const CircuitDev &c = p.circuit;
    const unsigned grid = (unsigned)(p.ldb / kCircW);
    if (grid == 0) return MP_OK;
    // A chain of more 8-column chunks than SMs runs on 16-column chunks, one
    // CTA per SM with the circuit in global memory, where that image fits:
    // the columns spread over the SMs more evenly than two 8-column CTAs to
    // some SMs and one to others, and a lane's entry indices serve twice the
    // columns.
    const size_t wide = circuit_image_bytes(c.Nh, 16) + kCircBarBytes;
    const bool aligned_out = a.user_ld % 8 == 0 && a.user_ld >= p.ldb;  // staged rows: one store per piece
    if (chain && (!user_out || aligned_out) && grid > (unsigned)di.sms && p.ldb % 16 == 0 &&
        wide + 1024 <= di.smem_optin) {
        auto *kern = circuit_step_kernel<true, true, 16>;
        MP_TRY(circuit_attr(kern, 6, true, wide, di));
        if (width) *width = 16;
        return circuit_kick(kern, a, (unsigned)(p.ldb / 16), wide, s);
    }
    // the circuit in global memory where the grid is larger than the SMs and
    // two images fit an SM but not two images with their circuits (a chain
    // writing full powers in rows of N entries keeps the circuit on chip:
    // its narrow stores, not its barriers, bound it)
    const size_t image = circuit_image_bytes(c.Nh, kCircW) + kCircBarBytes;
    const bool gblob = grid > (unsigned)di.sms && (!user_out || aligned_out) &&
                       2 * (image + 1024) <= di.smem_sm && 2 * (image + c.meta_bytes + 1024) > di.smem_sm;
    const size_t smem = image + (gblob ? 0 : c.meta_bytes);
    if (smem > di.smem_optin) return set_error(MP_EINVAL, "circuit does not fit shared memory");
    auto *kern = gblob ? (chain ? circuit_step_kernel<true, true, kCircW> : circuit_step_kernel<false, true, kCircW>)
                       : (chain ? circuit_step_kernel<true, false, kCircW> : circuit_step_kernel<false, false, kCircW>);
    MP_TRY(circuit_attr(kern, (chain ? 1 : 0) + (gblob ? 2 : 0), gblob, smem, di));
    if (width) *width = kCircW;
    return circuit_kick(kern, a, grid, smem, s);
}

int circuit_multi_chain(const PlanDev *const *plans, const uint16_t *const *B1, int count, int k_max,
                        int32_t *const *gdiag, cudaStream_t s) {
    if (count < 1 || count > kMultiChains) return set_error(MP_EINVAL, "%d chains in one launch", count);
    if (k_max < 2) return MP_OK;
    DeviceInfo di;
    MP_TRY(device_info(&di));
    MultiCircArgs m;
    memset(&m, 0, sizeof(m));
    m.count = count;
    // 16-column chunks where the first (longest) chain has more 8-column
    // chunks than the GPU has SMs and the widest image fits (as for one chain)
    size_t wide_max = 0;
    bool wide = plans[0]->ldb / kCircW > di.sms;
    for (int i = 0; i < count; ++i) {
        wide = wide && plans[i]->ldb % 16 == 0;
        wide_max = std::max(wide_max, circuit_image_bytes(plans[i]->circuit.Nh, 16) + kCircBarBytes);
    }
    wide = wide && wide_max + 1024 <= di.smem_optin;
    const int W = wide ? 16 : kCircW;
    size_t image_max = 0, meta_max = 0;
    int64_t total = 0;
    for (int i = 0; i < count; ++i) {
        const PlanDev &p = *plans[i];
        MP_TRY(circuit_args(p, B1[i], nullptr, k_max, nullptr, 0, 0, gdiag[i], 0, 1, &m.c[i]));
        m.chunks[i] = (int)(p.ldb / W);
        total += m.chunks[i];
        image_max = std::max(image_max, circuit_image_bytes(p.circuit.Nh, W) + kCircBarBytes);
        meta_max = std::max(meta_max, (size_t)p.circuit.meta_bytes + circuit_image_bytes(p.circuit.Nh, W) +
                                          kCircBarBytes);
    }
    if (total == 0) return MP_OK;
    const bool gblob = wide || (total > di.sms && 2 * (image_max + 1024) <= di.smem_sm);
    // The first chain takes one CTA per chunk, in as many waves of resident
    // CTAs as it needs (and room for one CTA of every other chain); the
    // others take the fewest chunks per CTA that fit them into those waves.
    const int64_t slots = (int64_t)di.sms * (gblob && 2 * (image_max + 1024) <= di.smem_sm ? 2 : 1);
    const int64_t room = (m.chunks[0] + count - 1 + slots - 1) / slots * slots;
    int f = 1;
    for (;;) {
        int64_t need = m.chunks[0];
        bool last = true;
        for (int i = 1; i < count; ++i) {
            need += (m.chunks[i] + f - 1) / f;
            last = last && f >= m.chunks[i];
        }
        if (need <= room || last) break;
        ++f;
    }
    for (int i = 0; i < count; ++i)
        m.cta0[i + 1] = m.cta0[i] + (i == 0 ? m.chunks[0] : (m.chunks[i] + f - 1) / f);
    const unsigned grid = (unsigned)m.cta0[count];
    const size_t smem = gblob ? image_max : meta_max;
    if (smem > di.smem_optin) return set_error(MP_EINVAL, "circuit does not fit shared memory");
    if (wide) {
        auto *kern = circuit_multi_kernel<true, 16>;
        MP_TRY(circuit_attr(kern, 7, true, smem, di));
        return circuit_kick(kern, m, grid, smem, s);
    }
    auto *kern = gblob ? circuit_multi_kernel<true, kCircW> : circuit_multi_kernel<false, kCircW>;
    MP_TRY(circuit_attr(kern, 4 + (gblob ? 1 : 0), gblob, smem, di));
    return circuit_kick(kern, m, grid, smem, s);
}

int circuit_step(const PlanDev &p, const uint16_t *Bin, uint16_t *Bout, int16_t *user_out,
                 int32_t *gdiag, cudaStream_t s) {
    return circuit_launch(p, false, Bin, Bout, 2, user_out, 0, gdiag, s);
}

// Failure injection: one step whose circuit copy expects 16 bytes that no
// copy sends, so every CTA's bounded wait runs out, latches MP_ETIMEOUT and
// the CTA returns (after a second bounded wait) without writing anything.
// The real copies are issued before the wait and land long before it ends.
int circuit_timeout_probe(const PlanDev &p, const uint16_t *Bin, uint16_t *Bout, cudaStream_t s) {
    return circuit_launch(p, false, Bin, Bout, 2, nullptr, 0, nullptr, s, 16);
}

int circuit_chain(const PlanDev &p, const uint16_t *B1, int k_max, int16_t *powers, size_t slot,
                  int32_t *gdiag, cudaStream_t s, int out_k0, int64_t powers_ld) {
    if (k_max < 2) return MP_OK;
    const int64_t ld = powers_ld ? powers_ld : p.N;
    if (powers && slot < (size_t)p.N * (size_t)ld) return set_error(MP_EINVAL, "power slots too small");
    return circuit_launch(p, true, B1, nullptr, k_max, powers, slot, gdiag, s, 0, out_k0, ld);
}

int circuit_chain_staged(const PlanDev &p, const uint16_t *B1, int k_max, int16_t *stage, size_t slot,
                         int32_t *gdiag, cudaStream_t s, int *width) {
    if (k_max < 2) return MP_OK;
    return circuit_launch(p, true, B1, nullptr, k_max, stage, slot, gdiag, s, 0, 1, p.ldb, width);
}

}  // namespace mp
