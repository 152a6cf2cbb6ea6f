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
// at most 64) so that the union U of the rows they gather stays small; the
// columns are cut into chunks of 64.  A work item is (group, chunk).  A
// persistent CTA walks its items; for each it streams the U rows' 64-column
// segments (128 B each) into shared memory with 1-D TMA bulk copies that
// complete on an mbarrier, double-buffered so the copies of the next item
// overlap the arithmetic of the current one.  A U list longer than one
// buffer is cut into stages, and the per-row minima carry over in
// registers.  Each warp owns rows of the group; its 32 lanes own the 64
// columns as 16-bit pairs, so every shared-memory read of a gathered row is
// one conflict-free 128-byte wavefront and the gather index is uniform
// across the warp.  Rows of the next power go to a padded internal buffer
// (and, when asked, to the caller's power array); the diagonal entries are
// min-reduced per item in shared memory and folded into g[k] with one
// atomicMin.
#include <algorithm>
#include <cstring>
#include <unordered_map>

#include "mp_internal.cuh"
#include "spmm.cuh"

namespace mp {

namespace {

constexpr int kThreads = 512;  // 16 warps
constexpr int kWarps = kThreads / 32;
constexpr int kGroupMax = 64;  // rows per group: at most 4 per warp
constexpr int kRowsPerWarp = kGroupMax / kWarps;
constexpr int kChunk = 64;     // columns per work item
constexpr int kRowBytes = kChunk * 2;
constexpr int kHeader = 128;   // barriers and per-item scratch ahead of the buffers

// ---------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Bounded wait: false when kSpinLimit polls pass without the phase flipping.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ uint32_t lds32(const uint8_t *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}

// Warp 0 streams the U rows of stage s (columns of chunk) into buf.
__device__ __forceinline__ void issue_stage(const SpStepArgs &a, int64_t chunk, int s,
                                            uint8_t *buf, uint64_t *bar, int lane) {
    const int u0 = a.stage_u0[s], u1 = a.stage_u0[s + 1];
    if (lane == 0) mbar_expect_tx(bar, (uint32_t)(u1 - u0) * kRowBytes);
    __syncwarp();
    const uint16_t *base = a.Bin + chunk * kChunk;
    for (int u = u0 + lane; u < u1; u += 32)
        tma_load_1d(buf + (size_t)(u - u0) * kRowBytes, base + (int64_t)a.urows[u] * a.ldb,
                    kRowBytes, bar);
}

template <bool kColConst>
__global__ void __launch_bounds__(kThreads, 1) sparse_step_kernel(SpStepArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    int32_t *dmin = reinterpret_cast<int32_t *>(smem + 16);
    uint8_t *bufs = smem + kHeader;
    const size_t buf_bytes = (size_t)a.cap_rows * kRowBytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // the last row of each buffer is the padding row: larger than any value
    if (threadIdx.x < 64) {
        uint8_t *infrow = bufs + (threadIdx.x >> 5) * buf_bytes + (size_t)(a.cap_rows - 1) * kRowBytes;
        reinterpret_cast<uint32_t *>(infrow)[lane] = 0xFFFFFFFFu;
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        dmin[0] = dmin[1] = (int32_t)kInf16;
        fence_barrier_init();
    }
    __syncthreads();

    const int64_t total = (int64_t)a.ngroups * a.nchunks;
    int64_t w = blockIdx.x;
    if (w >= total) return;
    int g = (int)(w % a.ngroups);
    int s = a.grp_stage0[g], s_end = a.grp_stage0[g + 1];
    if (warp == 0) issue_stage(a, w / a.ngroups, s, bufs, &bar[0], lane);

    uint32_t acc[kRowsPerWarp];
    uint32_t phases = 0;
    int unit = 0, item = 0;
    while (true) {
        const int b = unit & 1;
        // the next unit: the next stage of this item, or the first of the next item
        int64_t wn = w;
        int gn = g, sn = s + 1, sn_end = s_end;
        if (sn >= s_end) {
            wn = w + gridDim.x;
            if (wn < total) {
                gn = (int)(wn % a.ngroups);
                sn = a.grp_stage0[gn];
                sn_end = a.grp_stage0[gn + 1];
            }
        }
        const bool has_next = wn < total;
        if (has_next && warp == 0)
            issue_stage(a, wn / a.ngroups, sn, bufs + (b ^ 1) * buf_bytes, &bar[b ^ 1], lane);

        bool ok = mbar_wait_bounded(&bar[b], (phases >> b) & 1u);
        phases ^= 1u << b;
        if (__syncthreads_or(!ok)) {
            // a copy never landed: latch the error, let the other buffer's copy
            // (if any) finish so nothing writes shared memory after exit, return
            if (threadIdx.x == 0) atomicExch(a.status, MP_ETIMEOUT);
            if (has_next) mbar_wait_bounded(&bar[b ^ 1], (phases >> (b ^ 1)) & 1u);
            return;
        }

        const int64_t chunk = w / a.ngroups;
        const int64_t c0 = chunk * kChunk;
        const int row0 = a.grp_row0[g], nrows = a.grp_row0[g + 1] - row0;
        const bool first = (s == a.grp_stage0[g]), last = (s + 1 == s_end);
        const int eb = a.stage_ebase[s];
        const uint8_t *sb = bufs + b * buf_bytes + lane * 4;

#pragma unroll
        for (int ri = 0; ri < kRowsPerWarp; ++ri) {
            const int r = warp + ri * kWarps;
            if (first) acc[ri] = kInf16x2;
            if (r >= nrows) continue;
            const int e0 = a.stage_e[eb + r], e1 = a.stage_e[eb + r + 1];
            const uint4 *E = reinterpret_cast<const uint4 *>(a.ent + e0);
            if (kColConst) {
                uint32_t m0 = 0xFFFFFFFFu, m1 = 0xFFFFFFFFu;
                for (int t = 0; t < (e1 - e0) >> 3; ++t) {
                    const uint4 p = __ldg(E + 2 * t), q = __ldg(E + 2 * t + 1);
                    const uint32_t v0 = lds32(sb + p.x), v1 = lds32(sb + p.y);
                    const uint32_t v2 = lds32(sb + p.z), v3 = lds32(sb + p.w);
                    const uint32_t v4 = lds32(sb + q.x), v5 = lds32(sb + q.y);
                    const uint32_t v6 = lds32(sb + q.z), v7 = lds32(sb + q.w);
                    m0 = __vimin3_u16x2(m0, v0, v1);
                    m1 = __vimin3_u16x2(m1, v2, v3);
                    m0 = __vimin3_u16x2(m0, v4, v5);
                    m1 = __vimin3_u16x2(m1, v6, v7);
                }
                acc[ri] = __vimin3_u16x2(acc[ri], m0, m1);
            } else {
                uint32_t m = acc[ri];
                // two entries (offset, label pair) per 16-byte load, four per iteration
                for (int t = 0; t < (e1 - e0) >> 3; ++t) {
                    const uint4 p = __ldg(E + 2 * t), q = __ldg(E + 2 * t + 1);
                    m = __viaddmin_u16x2(lds32(sb + p.x), p.y, m);
                    m = __viaddmin_u16x2(lds32(sb + p.z), p.w, m);
                    m = __viaddmin_u16x2(lds32(sb + q.x), q.y, m);
                    m = __viaddmin_u16x2(lds32(sb + q.z), q.w, m);
                }
                acc[ri] = m;
            }
            if (last) {
                const int64_t q = row0 + r;
                const uint32_t v = acc[ri];  // = min(INF, .) since acc started at INF
                const uint32_t keep = kColConst ? v + (uint32_t)a.z[q] * 0x10001u : v;
                *reinterpret_cast<uint32_t *>(a.Bout + q * a.ldb + c0 + 2 * lane) = keep;
                const int64_t c = c0 + 2 * lane;
                if (a.user_out) {
                    int16_t *orow = a.user_out + q * a.N;
                    if (c < a.N) orow[c] = (int16_t)(v & 0xFFFFu);
                    if (c + 1 < a.N) orow[c + 1] = (int16_t)(v >> 16);
                }
                if (a.gdiag && q >= c0 && q < c0 + kChunk && lane == (int)((q - c0) >> 1))
                    atomicMin(&dmin[item & 1], (int32_t)(((q - c0) & 1) ? (v >> 16) : (v & 0xFFFFu)));
            }
        }
        __syncthreads();
        if (last) {
            if (threadIdx.x == 0) {
                const int32_t d = dmin[item & 1];
                if (a.gdiag && d < (int32_t)kInf16) atomicMin(a.gdiag, d);
                dmin[item & 1] = (int32_t)kInf16;
            }
            ++item;
        }
        ++unit;
        if (!has_next) break;
        w = wn;
        g = gn;
        s = sn;
        s_end = sn_end;
    }
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
__global__ void init_from_csr_kernel(const int64_t *__restrict__ row_ptr,
                                     const int32_t *__restrict__ col, const int16_t *__restrict__ val,
                                     int64_t N, int64_t ldb, const uint16_t *__restrict__ z,
                                     uint16_t *__restrict__ B, int16_t *__restrict__ user0,
                                     int32_t *__restrict__ g0) {
    const int64_t q = blockIdx.x;
    const uint16_t zq = z ? z[q] : 0;
    for (int64_t c = threadIdx.x; c < ldb; c += blockDim.x) {
        B[q * ldb + c] = (uint16_t)(kInf16 + zq);
        if (user0 && c < N) user0[q * N + c] = (int16_t)kInf16;
    }
    __syncthreads();  // the whole row is INF before the arcs land (one block per row)
    for (int64_t e = row_ptr[q] + threadIdx.x; e < row_ptr[q + 1]; e += blockDim.x) {
        const int64_t p = col[e];
        const uint32_t v = (uint32_t)(uint16_t)val[e];
        B[q * ldb + p] = (uint16_t)(v + zq);
        if (user0) user0[q * N + p] = (int16_t)v;
        if (g0 && p == q) atomicMin(g0, (int32_t)v);
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

int plan_build_host(const HostCsr &csr, bool colconst, const std::vector<uint16_t> &z,
                    int cap_rows, PlanHost *out) {
    const int64_t N = csr.N;
    const int umax = cap_rows - 1;  // the last buffer row is the INF padding row
    if (umax < 1) return set_error(MP_EINVAL, "shared-memory buffer too small");
    PlanHost &P = *out;
    P = PlanHost();
    P.N = N;
    P.colconst = colconst;
    P.cap_rows = cap_rows;
    P.z = z;
    if (P.z.size() != (size_t)N) P.z.assign((size_t)N, 0);
    P.ldb = ((N + kChunk - 1) / kChunk) * kChunk;
    P.nchunks = (int)(P.ldb / kChunk);
    P.nnz = csr.row_ptr[N];

    std::vector<int32_t> stamp((size_t)N, -1), local((size_t)N, -1);
    P.grp_row0.push_back(0);
    P.grp_stage0.push_back(0);
    P.stage_u0.push_back(0);
    int32_t gid = 0;
    int64_t q = 0;
    const int per_entry = colconst ? 1 : 2;  // 32-bit words per entry
    const int pad_to = colconst ? 8 : 4;     // entries per unrolled iteration
    while (q < N) {
        // grow the group while the union of gathered rows fits one buffer
        const int64_t g0 = q;
        int64_t ucount = 0;
        while (q < N && q - g0 < kGroupMax) {
            int64_t add = 0;
            for (int64_t e = csr.row_ptr[q]; e < csr.row_ptr[q + 1]; ++e)
                if (stamp[csr.col[e]] != gid) ++add;
            if (q > g0 && ucount + add > umax) break;
            for (int64_t e = csr.row_ptr[q]; e < csr.row_ptr[q + 1]; ++e)
                if (stamp[csr.col[e]] != gid) stamp[csr.col[e]] = gid;
            ucount += add;
            ++q;
        }
        // the union, sorted, cut into stages of at most umax rows
        std::vector<int32_t> U;
        U.reserve((size_t)ucount);
        for (int64_t r = g0; r < q; ++r)
            for (int64_t e = csr.row_ptr[r]; e < csr.row_ptr[r + 1]; ++e)
                if (local[csr.col[e]] != gid) {
                    local[csr.col[e]] = gid;
                    U.push_back(csr.col[e]);
                }
        std::sort(U.begin(), U.end());
        std::vector<int32_t> where((size_t)U.size());
        const int nst = U.empty() ? 1 : (int)((U.size() + umax - 1) / umax);
        for (int st = 0; st < nst; ++st) {
            const size_t ub = (size_t)st * umax, ue = std::min(U.size(), ub + (size_t)umax);
            for (size_t u = ub; u < ue; ++u) P.urows.push_back(U[u]);
            P.stage_u0.push_back((int32_t)P.urows.size());
            P.stage_ebase.push_back((int32_t)P.stage_e.size());
            for (int64_t r = g0; r < q; ++r) {
                P.stage_e.push_back((int32_t)(P.ent.size() / per_entry));
                // entries of row r whose gathered row falls in this stage, by U order
                std::vector<std::pair<int32_t, uint32_t>> es;
                for (int64_t e = csr.row_ptr[r]; e < csr.row_ptr[r + 1]; ++e) {
                    const int32_t p = csr.col[e];
                    const size_t u = (size_t)(std::lower_bound(U.begin(), U.end(), p) - U.begin());
                    if (u < ub || u >= ue) continue;
                    es.push_back({(int32_t)(u - ub), (uint32_t)(uint16_t)csr.val[e]});
                }
                std::sort(es.begin(), es.end());
                while (es.size() % pad_to) es.push_back({umax, colconst ? 0u : 0u});
                for (auto &pr : es) {
                    // the padding row sits at index cap_rows - 1 = umax
                    P.ent.push_back((uint32_t)pr.first * kRowBytes);
                    if (!colconst) P.ent.push_back(pr.second * 0x10001u);
                }
            }
            P.stage_e.push_back((int32_t)(P.ent.size() / per_entry));
        }
        P.grp_row0.push_back((int32_t)q);
        P.grp_stage0.push_back((int32_t)(P.stage_u0.size() - 1));
        ++gid;
    }
    P.ngroups = gid;
    // entry indices are in units of entries; convert to 32-bit word offsets
    if (!colconst)
        for (auto &v : P.stage_e) v *= 2;
    return MP_OK;
}

int plan_upload(const PlanHost &h, PlanDev *d, cudaStream_t s, bool persistent) {
    d->N = h.N;
    d->ldb = h.ldb;
    d->ngroups = h.ngroups;
    d->nchunks = h.nchunks;
    d->cap_rows = h.cap_rows;
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
    MP_TRY(up(d->stage_ebase, h.stage_ebase.data(), h.stage_ebase.size() * 4));
    MP_TRY(up(d->stage_e, h.stage_e.data(), h.stage_e.size() * 4));
    MP_TRY(up(d->urows, h.urows.data(), h.urows.size() * 4));
    MP_TRY(up(d->ent, h.ent.data(), h.ent.size() * 4));
    MP_TRY(up(d->z, h.z.data(), h.z.size() * 2));
    d->h2d_bytes = (h.grp_row0.size() + h.grp_stage0.size() + h.stage_u0.size() +
                    h.stage_ebase.size() + h.stage_e.size() + h.urows.size() + h.ent.size()) * 4 +
                   h.z.size() * 2;
    return MP_OK;
}

int sparse_cap_rows(int *cap_rows, int *blocks_per_sm) {
    DeviceInfo di;
    MP_TRY(device_info(&di));
    // one CTA per SM, two buffers of cap_rows rows of 128 B
    size_t budget = di.smem_optin - 1024 - kHeader;
    int cap = (int)(budget / (2 * (size_t)kRowBytes));
    if (cap > 2048) cap = 2048;
    *cap_rows = cap;
    *blocks_per_sm = 1;
    return MP_OK;
}

int sparse_step(const PlanDev &p, const uint16_t *Bin, uint16_t *Bout, int16_t *user_out,
                int32_t *gdiag, cudaStream_t s) {
    DeviceInfo di;
    MP_TRY(device_info(&di));
    int *status = nullptr;
    MP_TRY(device_status_ptr(&status));
    SpStepArgs a;
    memset(&a, 0, sizeof(a));
    a.grp_row0 = p.grp_row0.as<int32_t>();
    a.grp_stage0 = p.grp_stage0.as<int32_t>();
    a.stage_u0 = p.stage_u0.as<int32_t>();
    a.stage_ebase = p.stage_ebase.as<int32_t>();
    a.stage_e = p.stage_e.as<int32_t>();
    a.urows = p.urows.as<int32_t>();
    a.ent = p.ent.as<uint32_t>();
    a.z = p.z.as<uint16_t>();
    a.ngroups = p.ngroups;
    a.nchunks = p.nchunks;
    a.cap_rows = p.cap_rows;
    a.N = p.N;
    a.ldb = p.ldb;
    a.Bin = Bin;
    a.Bout = Bout;
    a.user_out = user_out;
    a.gdiag = gdiag;
    a.status = status;
    const size_t smem = kHeader + 2 * (size_t)p.cap_rows * kRowBytes;
    const int64_t total = (int64_t)p.ngroups * p.nchunks;
    int64_t grid = std::min<int64_t>(total, (int64_t)di.sms);
    if (grid < 1) return MP_OK;
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
    if (p.colconst)
        sparse_step_kernel<true><<<(unsigned)grid, kThreads, smem, s>>>(a);
    else
        sparse_step_kernel<false><<<(unsigned)grid, kThreads, smem, s>>>(a);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int sparse_init_from_dense(const PlanDev &p, const int16_t *A, uint16_t *B0, int16_t *user0,
                           int32_t *g0, cudaStream_t s) {
    dim3 grid((unsigned)p.N, (unsigned)std::min<int64_t>((p.ldb + 255) / 256, 64));
    init_from_dense_kernel<<<grid, 256, 0, s>>>(A, p.N, p.ldb, p.colconst ? p.z.as<uint16_t>() : nullptr,
                                                B0, user0, g0);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int sparse_init_from_csr(const PlanDev &p, const int64_t *row_ptr, const int32_t *col,
                         const int16_t *val, uint16_t *B0, int16_t *user0, int32_t *g0,
                         cudaStream_t s) {
    // one block per row so the INF fill precedes the arc scatter within the block
    dim3 grid((unsigned)p.N, 1);
    init_from_csr_kernel<<<grid, 256, 0, s>>>(row_ptr, col, val, p.N, p.ldb,
                                              p.colconst ? p.z.as<uint16_t>() : nullptr, B0, user0, g0);
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
