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
// reads at n = 9 about 6.7 rows per output row instead of the 88 arcs of a
// row: 23271 row reads per column against nnz(A) = 303097.  The result is
// the same minimum, bit for bit.
//
// Host: successor sets as bitsets; for each row, in order of set size, the
// rows whose sets it contains, then the greedy cover (take the candidate
// covering most of what is still uncovered while it covers at least two).
// A row's level is one more than the deepest row of its cover.  Each level's
// rows, longest list first, are cut into slices of one warp's rows; a slice
// stores its lists in blocks of 8 row indices per row (16 bytes, one load
// per lane for 8 entries; a short list is padded with the INF row).
//
// Device (circuit_step_kernel): one CTA per chunk of W columns.  The circuit
// (one blob, the same for every chunk and every step) is copied into shared
// memory while the previous step finishes; then the chunk of X (N rows of W
// columns).  The levels run in order with a block barrier between them,
// touching only shared memory: a warp takes every 16th slice of a level,
// each lane (or lane pair at W = 16) one row, 16 bytes of it per lane.  A
// row's result goes to shared memory for the later levels and, with its
// label added, straight to the next buffer; the diagonal entries are
// min-reduced and folded into g[k].
#include <algorithm>
#include <cstring>
#include <mutex>

#include "mp_internal.cuh"
#include "spmm.cuh"

namespace mp {

namespace {

#ifndef MP_CIRC_THREADS
#define MP_CIRC_THREADS 512
#endif
constexpr int kCircThreads = MP_CIRC_THREADS;
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
__device__ __forceinline__ uint2 clds_v2(uint32_t addr) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
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
    uint32_t meta_bytes, off_slices, off_rowinfo, off_first, off_ents, off_z;
    int levels;
    int k_max;            // a chain: P_2 .. P_{k_max}
    int16_t *user_out;    // the caller's power(s), or null
    size_t slot;          // a chain: entries between the caller's powers
    int32_t *gdiag;       // one step: g[k]; a chain: g[0 .. k_max - 1]
    int *status;
    uint32_t extra_tx;    // bytes expected beyond the circuit's (0; > 0 only to inject a timeout)
};

__device__ __forceinline__ uint32_t pick_word(const uint4 &v, int k) {
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

// acc = min(acc, the image rows an entry block names), 16 bytes per lane;
// entries naming the INF row (the padding of short lists, index 2Nh) load
// nothing, the others live at image row (index + sh) mod 2Nh.
template <int RB>
__device__ __forceinline__ void fold8(uint4 &acc, const uint4 &e, uint32_t rbase, uint32_t N2,
                                      uint32_t sh) {
    const uint32_t ix[8] = {e.x & 0xFFFFu, e.x >> 16, e.y & 0xFFFFu, e.y >> 16,
                            e.z & 0xFFFFu, e.z >> 16, e.w & 0xFFFFu, e.w >> 16};
    uint4 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        uint32_t j = ix[k] + sh;
        if (j >= N2) j -= N2;
        v[k] = ix[k] != N2 ? clds_v4(rbase + j * RB) : make_uint4(~0u, ~0u, ~0u, ~0u);
    }
    acc.x = __vimin3_u16x2(__vimin3_u16x2(acc.x, v[0].x, v[1].x), __vimin3_u16x2(v[2].x, v[3].x, v[4].x),
                           __vimin3_u16x2(v[5].x, v[6].x, v[7].x));
    acc.y = __vimin3_u16x2(__vimin3_u16x2(acc.y, v[0].y, v[1].y), __vimin3_u16x2(v[2].y, v[3].y, v[4].y),
                           __vimin3_u16x2(v[5].y, v[6].y, v[7].y));
    acc.z = __vimin3_u16x2(__vimin3_u16x2(acc.z, v[0].z, v[1].z), __vimin3_u16x2(v[2].z, v[3].z, v[4].z),
                           __vimin3_u16x2(v[5].z, v[6].z, v[7].z));
    acc.w = __vimin3_u16x2(__vimin3_u16x2(acc.w, v[0].w, v[1].w), __vimin3_u16x2(v[2].w, v[3].w, v[4].w),
                           __vimin3_u16x2(v[5].w, v[6].w, v[7].w));
}

// Shared memory of a step: the image (X, result, INF row), then the circuit,
// then its copies' mbarrier.
__host__ __device__ __forceinline__ size_t circuit_image_bytes(int64_t N, int W) {
    return ((size_t)(2 * N + 1) * (size_t)(2 * W) + 15) & ~(size_t)15;
}
constexpr uint32_t kCircBarBytes = 16;
constexpr uint32_t kMetaCopy = 32768;  // bytes per bulk copy of the circuit

// W columns per CTA; a row is 2W bytes, read by W / 8 lanes (16 bytes each).
// One step (kChain false): X from Bin, the result (labelled) to Bout.  A
// chain (kChain true): the CTA runs every step of the chain on its chunk
// without leaving the SM -- column chunk c of P_{k+1} depends only on chunk c
// of P_k -- so after a step the result region, with the labels added in
// place, is the next step's X, and the two regions swap: with sh = 0 or N,
// image index j (X rows 0..N-1, result rows Nh..Nh+N-1, Nh = N rounded up to
// 8) lives at (j + sh) mod 2Nh, sh = 0 or Nh.
template <int W, bool kChain>
__global__ void __launch_bounds__(kCircThreads, 1) circuit_step_kernel(CircArgs a) {
    constexpr int LPR = W / 8;       // lanes per row
    constexpr int SR = 32 / LPR;     // rows per slice
    constexpr int RB = 2 * W;        // bytes per row
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t sbase = csmem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t N = a.N;
    const uint32_t Nh = (uint32_t)a.Nh, N2 = 2 * Nh;
    const int64_t c0 = (int64_t)blockIdx.x * W;
    const uint32_t mb = sbase + (uint32_t)circuit_image_bytes(Nh, W);
    __shared__ int32_t s_dmin;

    // The circuit: plan data only, so its bulk copies start before the
    // previous step has finished.  The barrier's initialisation is made
    // visible to the other threads by the block barrier below, before any of
    // them waits on it.
    const uint32_t bar = mb + a.meta_bytes;
    if (threadIdx.x == 0) {
        s_dmin = (int32_t)kInf16;
        cmbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        cmbar_arrive_expect_tx(bar, a.meta_bytes + a.extra_tx);
        for (uint32_t o = 0; o < a.meta_bytes; o += kMetaCopy)
            cbulk_copy(mb + o, a.meta + o, min(kMetaCopy, a.meta_bytes - o), bar);
    }
    // row 2Nh of the image: above every value, the padding of short lists
    if (threadIdx.x < RB / 4) reinterpret_cast<uint32_t *>(smem + (size_t)N2 * RB)[threadIdx.x] = 0xFFFFFFFFu;
    // Programmatic dependent launch: the previous step's output (our X) is
    // read only after its grid has completed.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // X's chunk: N rows of RB bytes, in 16-byte pieces
    for (int64_t pc = threadIdx.x; pc < N * LPR; pc += kCircThreads) {
        const int64_t r = pc / LPR;
        const int part = (int)(pc - r * LPR);
        ccp_async16(sbase + (uint32_t)(r * RB + part * 16), a.Bin + r * a.ldb + c0 + part * 8);
    }
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

    const int i = lane / LPR, h = lane % LPR;
    const uint32_t hb = (uint32_t)h * 16;
    const int64_t col0 = c0 + (int64_t)h * 8;
    const uint32_t m_sl = mb + a.off_slices, m_ri = mb + a.off_rowinfo;
    const uint32_t m_fi = mb + a.off_first, m_en = mb + a.off_ents;
    const int k_last = kChain ? a.k_max : 2;
    uint32_t sh = 0;
    for (int k = 2; k <= k_last; ++k) {
        int32_t dmin = (int32_t)kInf16;
        for (int l = 0; l < a.levels; ++l) {
            const int s1 = (int)clds_u32(mb + 4u * (uint32_t)(l + 1));
            for (int s = (int)clds_u32(mb + 4u * (uint32_t)l) + warp; s < s1; s += kCircWarps) {
                const uint32_t slot = (uint32_t)s * SR + (uint32_t)i;
                const uint2 d = clds_v2(m_sl + 8u * (uint32_t)s);
                const uint2 ri = clds_v2(m_ri + 8u * slot);
                uint4 acc = make_uint4(kInf16x2, kInf16x2, kInf16x2, kInf16x2);
                fold8<RB>(acc, clds_v4(m_fi + 16u * slot), sbase + hb, N2, sh);
                // the few rows longer than one block: their later blocks
                for (uint32_t jb = 1; jb < d.y; ++jb)
                    fold8<RB>(acc, clds_v4(m_en + 16u * (d.x + (jb - 1) * SR + (uint32_t)i)), sbase + hb,
                              N2, sh);
                const uint32_t q = ri.x & 0xFFFFu;
                if (q == 0xFFFFu) continue;
                // the result row, for the later levels (and the next step)
                uint32_t rr = Nh + q + sh;
                if (rr >= N2) rr -= N2;
                csts_v4(sbase + rr * RB + hb, acc);
                if (!kChain) {
                    const uint32_t zq = (ri.x >> 16) * 0x10001u;
                    *reinterpret_cast<uint4 *>(a.Bout + (int64_t)q * a.ldb + col0) =
                        make_uint4(acc.x + zq, acc.y + zq, acc.z + zq, acc.w + zq);
                }
                const uint32_t dc = ri.y & 0xFFFFu;
                if (a.gdiag && dc != 0xFFFFu && (int64_t)dc >= col0 && (int64_t)dc < col0 + 8) {
                    const int kk = (int)((int64_t)dc - col0);
                    const uint32_t wv = pick_word(acc, kk >> 1);
                    dmin = min(dmin, (int32_t)((kk & 1) ? wv >> 16 : wv & 0xFFFFu));
                }
                if (a.user_out) {
                    int16_t *orow = a.user_out + (kChain ? (size_t)(k - 1) * a.slot : 0) +
                                    (int64_t)(ri.y >> 16) * N;
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const uint32_t wv = pick_word(acc, kk >> 1);
                        if (col0 + kk < N) orow[col0 + kk] = (int16_t)((kk & 1) ? wv >> 16 : wv & 0xFFFFu);
                    }
                }
            }
            __syncthreads();  // this level's rows are read by the later levels
        }
        if (a.gdiag) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dmin = min(dmin, __shfl_xor_sync(0xFFFFFFFFu, dmin, o));
            if (lane == 0 && dmin < (int32_t)kInf16) atomicMin(&s_dmin, dmin);
        }
        if (kChain) {
            // the labels, in place: the result becomes the next step's X
            const uint32_t m_z = mb + a.off_z;
            for (int64_t pc = threadIdx.x; pc < N * LPR; pc += kCircThreads) {
                const uint32_t q = (uint32_t)(pc / LPR);
                const uint32_t part = (uint32_t)(pc - (int64_t)q * LPR);
                uint32_t rr = Nh + q + sh;
                if (rr >= N2) rr -= N2;
                const uint32_t addr = sbase + rr * RB + part * 16;
                const uint32_t zw = clds_u32(m_z + 4u * (q >> 1));
                const uint32_t zq = ((q & 1) ? zw >> 16 : zw & 0xFFFFu) * 0x10001u;
                const uint4 v = clds_v4(addr);
                csts_v4(addr, make_uint4(v.x + zq, v.y + zq, v.z + zq, v.w + zq));
            }
            sh = Nh - sh;
        }
        __syncthreads();
        if (threadIdx.x == 0 && a.gdiag) {
            const int32_t v = s_dmin;
            if (v < (int32_t)kInf16) atomicMin(kChain ? a.gdiag + (k - 1) : a.gdiag, v);
            s_dmin = (int32_t)kInf16;  // the next step's minima arrive after its levels
        }
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace

int circuit_cover_host(const HostCsr &csr, CircuitCover *out) {
    const int64_t N = csr.N;
    if (N < 1 || 2 * N + 1 > 0xFFFF) return set_error(MP_EINVAL, "N = %lld too large for a circuit", (long long)N);
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
            int64_t best = -1, bg = 1;
            size_t bi = 0;
            for (size_t k = 0; k < cand.size(); ++k) {
                const uint64_t *Sc = &S[(size_t)(cand[k] * nw)];
                int64_t g = 0;
                for (int64_t w = 0; w < nw; ++w) g += __builtin_popcountll(Sc[w] & U[(size_t)w]);
                if (g > bg) {
                    bg = g;
                    best = cand[k];
                    bi = k;
                }
            }
            if (best < 0) break;  // no candidate covers two or more: read the rest directly
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

int circuit_slice_host(const CircuitCover &cv, int W, CircuitHost *out) {
    if (W != 8 && W != 16) return set_error(MP_EINVAL, "circuit width %d", W);
    const int64_t N = cv.N;
    CircuitHost &C = *out;
    C = CircuitHost();
    C.N = N;
    C.Nh = (N + 7) & ~(int64_t)7;
    C.W = W;
    C.levels = cv.levels;
    C.reads = cv.reads;
    C.cover_reads = cv.cover_reads;
    // per level: rows longest list first, cut into slices of one warp's rows
    const int SR = 32 / (W / 8);
    if (2 * C.Nh + 1 > 0xFFFF) return set_error(MP_EINVAL, "N = %lld too large for a circuit", (long long)N);
    const uint16_t pad = (uint16_t)(2 * C.Nh);
    // a list entry in image rows: X rows stay, result row N + q' moves to Nh + q'
    auto img = [&](uint32_t v) { return v < (uint32_t)N ? v : v - (uint32_t)N + (uint32_t)C.Nh; };
    C.level_slice0.push_back(0);
    for (int l = 0; l < C.levels; ++l) {
        std::vector<int64_t> lr;
        for (int64_t q = 0; q < N; ++q)
            if (cv.level[(size_t)q] == l) lr.push_back(q);
        std::stable_sort(lr.begin(), lr.end(), [&](int64_t x, int64_t y) {
            return cv.lists[(size_t)x].size() > cv.lists[(size_t)y].size();
        });
        for (size_t r0 = 0; r0 < lr.size(); r0 += (size_t)SR) {
            const size_t r1 = std::min(lr.size(), r0 + (size_t)SR);
            const size_t len = cv.lists[(size_t)lr[r0]].size();
            const uint32_t nb = (uint32_t)std::max<size_t>(1, (len + 7) / 8);
            C.slices.push_back((uint32_t)(C.ents.size() / 8));
            C.slices.push_back(nb);
            for (int i = 0; i < SR; ++i)
                C.rows.push_back(r0 + (size_t)i < r1 ? (uint32_t)lr[r0 + (size_t)i] : 0xFFFFFFFFu);
            // Each list in an order of its own (min is order-free), chosen so
            // that at every entry position the loads spread over the
            // shared-memory banks.  An image row of 2W bytes sits in bank
            // group (row mod groups), groups = 128 / 2W; a 16-byte load is
            // served a quarter warp (8 lanes, so `groups` rows) at a time, and
            // a quarter takes as many passes as its fullest group.  Greedy:
            // position by position, each row of a quarter takes its remaining
            // entry whose group that quarter uses least so far.  The result
            // rows start at a multiple of 8, so the regions' swap in a chain
            // keeps every row's group.
            const int groups = 128 / (2 * W);
            std::vector<std::vector<uint32_t>> rem((size_t)SR);
            for (int i = 0; i < SR; ++i)
                if (r0 + (size_t)i < r1)
                    for (uint32_t v : cv.lists[(size_t)lr[r0 + (size_t)i]]) rem[(size_t)i].push_back(img(v));
            std::vector<uint16_t> blk((size_t)nb * SR * 8, pad);
            for (uint32_t j = 0; j < nb * 8; ++j) {
                std::vector<int> used((size_t)groups, 0);
                for (int i = 0; i < SR; ++i) {
                    if (i % groups == 0) std::fill(used.begin(), used.end(), 0);
                    auto &li = rem[(size_t)i];
                    if (li.empty()) continue;
                    size_t best = 0;
                    for (size_t t = 1; t < li.size(); ++t)
                        if (used[li[t] % groups] < used[li[best] % groups]) best = t;
                    ++used[li[best] % groups];
                    blk[((size_t)(j / 8) * SR + (size_t)i) * 8 + (j % 8)] = (uint16_t)li[best];
                    li.erase(li.begin() + (long)best);
                }
            }
            C.first.insert(C.first.end(), blk.begin(), blk.begin() + (size_t)SR * 8);
            C.ents.insert(C.ents.end(), blk.begin() + (size_t)SR * 8, blk.end());
        }
        C.level_slice0.push_back((int32_t)(C.slices.size() / 2));
    }
    return MP_OK;
}

int circuit_build_host(const HostCsr &csr, int W, CircuitHost *out) {
    CircuitCover cv;
    MP_TRY(circuit_cover_host(csr, &cv));
    return circuit_slice_host(cv, W, out);
}

// Section offsets of the circuit blob (bytes, each section a multiple of 16).
struct CircLayout {
    uint32_t sl = 0, ri = 0, fi = 0, en = 0, z = 0, total = 0;
};
static CircLayout circuit_layout(const CircuitHost &h) {
    auto r16 = [](size_t b) { return (uint32_t)((b + 15) & ~(size_t)15); };
    CircLayout L;
    L.sl = r16(h.level_slice0.size() * 4);
    L.ri = L.sl + r16(h.slices.size() * 4);     // two words per slice
    L.fi = L.ri + r16(h.rows.size() * 8);       // two words per slot
    L.en = L.fi + r16(h.first.size() * 2);
    L.z = L.en + r16(h.ents.size() * 2);
    L.total = L.z + r16((size_t)h.N * 2);       // the rows' labels
    return L;
}

int circuit_smem_bytes(const CircuitHost &h, size_t *bytes) {
    *bytes = circuit_image_bytes(h.Nh, h.W) + circuit_layout(h).total + kCircBarBytes;
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
        h.N != d->N)
        return set_error(MP_EINVAL, "circuit of the wrong size");
    if (d->ldb % h.W) return set_error(MP_EINVAL, "circuit width does not divide the buffer");
    const CircLayout L = circuit_layout(h);
    std::vector<uint8_t> blob(L.total, 0);
    memcpy(blob.data(), h.level_slice0.data(), h.level_slice0.size() * 4);
    memcpy(blob.data() + L.sl, h.slices.data(), h.slices.size() * 4);
    std::vector<uint32_t> ri(h.rows.size() * 2);
    for (size_t k = 0; k < h.rows.size(); ++k) {
        const uint32_t q = h.rows[k];
        if (q == 0xFFFFFFFFu) {
            ri[2 * k] = 0xFFFFu;
            ri[2 * k + 1] = 0xFFFFu;
            continue;
        }
        const int32_t dc = diagcol[q];
        if (z[q] > 0x7FFFu || dc >= 0xFFFF || caller[q] < 0 || caller[q] > 0xFFFF)
            return set_error(MP_EINVAL, "circuit row fields out of range");
        ri[2 * k] = q | ((uint32_t)z[q] << 16);
        ri[2 * k + 1] = (dc < 0 ? 0xFFFFu : (uint32_t)dc) | ((uint32_t)caller[q] << 16);
    }
    memcpy(blob.data() + L.ri, ri.data(), ri.size() * 4);
    memcpy(blob.data() + L.fi, h.first.data(), h.first.size() * 2);
    memcpy(blob.data() + L.en, h.ents.data(), h.ents.size() * 2);
    memcpy(blob.data() + L.z, z.data(), z.size() * 2);
    MP_TRY(c.meta.alloc(L.total ? L.total : 16, s, true));
    MP_CUDA_TRY(cudaMemcpyAsync(c.meta.p, blob.data(), L.total, cudaMemcpyHostToDevice, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));  // the host blob goes out of scope
    c.W = h.W;
    c.Nh = h.Nh;
    c.levels = h.levels;
    c.nslices = (int64_t)h.slices.size() / 2;
    c.meta_bytes = L.total;
    c.off_slices = L.sl;
    c.off_rowinfo = L.ri;
    c.off_first = L.fi;
    c.off_ents = L.en;
    c.off_z = L.z;
    c.ready = true;
    return MP_OK;
}

// One launch: a step (Bin -> Bout) or a whole chain from Bin = P_1.
static int circuit_launch(const PlanDev &p, bool chain, const uint16_t *Bin, uint16_t *Bout, int k_max,
                          int16_t *user_out, size_t slot, int32_t *gdiag, cudaStream_t s,
                          uint32_t extra_tx = 0) {
    const CircuitDev &c = p.circuit;
    if (!c.ready) return set_error(MP_EINVAL, "plan has no circuit");
    if (p.narrow && user_out) return set_error(MP_EINVAL, "a narrow chain has no full powers to write");
    DeviceInfo di;
    MP_TRY(device_info(&di));
    CircArgs a;
    memset(&a, 0, sizeof(a));
    a.Bin = Bin;
    a.Bout = Bout;
    a.N = p.N;
    a.Nh = c.Nh;
    a.ldb = p.ldb;
    a.meta = c.meta.as<uint8_t>();
    a.meta_bytes = c.meta_bytes;
    a.off_slices = c.off_slices;
    a.off_rowinfo = c.off_rowinfo;
    a.off_first = c.off_first;
    a.off_ents = c.off_ents;
    a.off_z = c.off_z;
    a.levels = c.levels;
    a.k_max = k_max;
    a.user_out = user_out;
    a.slot = slot;
    a.gdiag = gdiag;
    a.extra_tx = extra_tx;
    MP_TRY(device_status_ptr(&a.status));
    const size_t smem = circuit_image_bytes(c.Nh, c.W) + c.meta_bytes + kCircBarBytes;
    if (smem > di.smem_optin) return set_error(MP_EINVAL, "circuit does not fit shared memory");
    const unsigned grid = (unsigned)(p.ldb / c.W);
    if (grid == 0) return MP_OK;
    auto *kern = c.W == 16 ? (chain ? circuit_step_kernel<16, true> : circuit_step_kernel<16, false>)
                           : (chain ? circuit_step_kernel<8, true> : circuit_step_kernel<8, false>);
    // the dynamic size each kernel may take, raised as larger plans come
    static std::mutex attr_mu;
    static size_t attr_set[4][64] = {};
    const int kind = (c.W == 16 ? 0 : 2) + (chain ? 1 : 0);
    {
        std::lock_guard<std::mutex> lk(attr_mu);
        if (di.device >= 64 || attr_set[kind][di.device] < smem) {
            MP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            if (di.device < 64) attr_set[kind][di.device] = smem;
        }
    }
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
                  int32_t *gdiag, cudaStream_t s) {
    if (k_max < 2) return MP_OK;
    if (powers && slot < (size_t)p.N * (size_t)p.N) return set_error(MP_EINVAL, "power slots too small");
    return circuit_launch(p, true, B1, nullptr, k_max, powers, slot, gdiag, s);
}

}  // namespace mp
