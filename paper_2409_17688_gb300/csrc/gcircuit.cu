// K2 by a reuse circuit in global memory: the transfer step for path orders
// whose column chunk does not fit shared memory (n >= 10).
//
// The circuit is the one of circuit.cu: row q of A (x) X is the minimum
// over its successors p of z_p + X[p], and where the successors of q' are a
// subset of those of q, row q' of the result stands in for all of them.
// Here the subsets come from the arc rule itself rather than from a search
// over all pairs of rows (which is quadratic in N): the source word q
// enters the rule only through its 0-letters (each a zero next to the
// target's letter) and its 2-letters (each forcing a 0 in the target), so
// turning a 0 or 1 of q into a 2 gives a word q' with
// Out(q') = Out(q) n {p : p_i = 0}.  Row q's candidate covers are the
// correct words with one or two letters so turned, scored as in circuit.cu
// (arcs covered less kCircLambda per level added), and its direct reads are
// the successors no chosen cover holds.
//
// Device (gcircuit_kernel): one CTA per chunk of W = 8 L columns (L = 4,
// 8, 16 or 32 lanes per row, 16 bytes each), the whole chain in one launch:
// the chunk's rows of the previous power X and of the result R stay in the
// chain's two global buffers (L2 holds them where they fit), and every step
// computes the levels in order with a block barrier between them.  A warp
// task is 32 / L rows of one level, longest lists first; its lanes walk
// their row's list eight entries at a time, the eight row loads issued
// before any is folded (the kernel is bound by the latency of L2 and HBM).  The buffers hold the powers
// themselves, not labelled: an entry of a direct read carries its label and
// is folded with a fused add-min (__viaddmin_u16x2), a cover entry with a
// plain minimum.  After the levels the chunk's diagonal entries (at most W
// rows) are min-reduced into g[k], and full powers go to the caller's
// layout row by row.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "mp_internal.cuh"
#include "spmm.cuh"

namespace mp {

namespace {

constexpr int kGThreads = 512;
constexpr int kGWarps = kGThreads / 32;
// entry words: bits 0..23 the row; bit 31 a result row (cover); bit 30 a
// pad; bits 24..27 the label of a direct read
constexpr uint32_t kGCover = 0x80000000u, kGPad = 0x40000000u, kGRow = 0x00FFFFFFu;

struct GArgs {
    const uint16_t *B0;   // the first X (P_1 for a chain, P_k for one step)
    uint16_t *B1;         // the first R; a chain alternates the two
    int64_t N, ldb;       // ldb: the buffers' leading dimension (a block's width)
    int64_t col_base;     // plan column of the buffers' column 0 (column blocks)
    const uint32_t *level_task0;  // [levels + 1]
    const uint4 *tasks;           // per task, per row slot {row, off4, len4, task max len4}
    const uint4 *ents;            // four entries each
    const uint32_t *drow;         // per buffer column, the row with its diagonal entry there
    const int32_t *caller;        // per internal row, the caller's row
    int levels;
    int k_max, out_k0;
    int16_t *user_out;
    size_t slot;
    int32_t *gdiag;
    uint32_t nents4;      // blocks of four entries (bounds-checked builds)
    int *status;
};

// The 16 bytes an entry names (all ones for padding: above every value, so
// it never lowers a minimum) and the label to add.
__device__ __forceinline__ void gload(uint32_t e, const uint16_t *X, const uint16_t *R, int64_t ldb,
                                      int64_t col, uint4 &v, uint32_t &zz, int64_t N, int *status) {
    if (e & kGPad) {
        v = make_uint4(~0u, ~0u, ~0u, ~0u);
        zz = 0;
        return;
    }
    const bool cov = (e & kGCover) != 0;
    const int64_t row = mp_ix((int64_t)(e & kGRow), N, status);
    v = *reinterpret_cast<const uint4 *>((cov ? R : X) + row * ldb + col);
    zz = cov ? 0u : ((e >> 24) & 0xFu) * 0x10001u;
}
__device__ __forceinline__ void gmin(uint4 &acc, const uint4 &v, uint32_t zz) {
    acc.x = __viaddmin_u16x2(v.x, zz, acc.x);
    acc.y = __viaddmin_u16x2(v.y, zz, acc.y);
    acc.z = __viaddmin_u16x2(v.z, zz, acc.z);
    acc.w = __viaddmin_u16x2(v.w, zz, acc.w);
}

// One step (kChain false): X = B0, R = B1.  A chain: steps k = 2..k_max,
// X and R swapping between B0 and B1 (column chunk c of P_{k+1} depends only
// on chunk c of P_k, so each CTA runs its chunk through every step alone).
template <int L, bool kChain>
__global__ void __launch_bounds__(kGThreads, 2) gcircuit_kernel(GArgs a) {
    constexpr int W = 8 * L, RPT = 32 / L;  // columns per chunk, rows per warp task
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slotr = lane / L, part = lane % L;
    const int64_t cb = (int64_t)blockIdx.x * W;
    const int64_t col = cb + (int64_t)part * 8;
    const int64_t N = a.N, ldb = a.ldb;
    // the row whose diagonal entry lies in column cb + t (threads t < W)
    uint32_t drow = 0xFFFFFFFFu;
    if (a.gdiag && threadIdx.x < W) drow = a.drow[a.col_base + cb + threadIdx.x];
    if (drow != 0xFFFFFFFFu) drow = mp_ix(drow, (uint32_t)N, a.status);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const uint16_t *X = a.B0;
    uint16_t *R = a.B1;
    const int k_last = kChain ? a.k_max : 2;
    for (int k = 2; k <= k_last; ++k) {
        for (int l = 0; l < a.levels; ++l) {
            const int t1 = (int)a.level_task0[l + 1];
            for (int t = (int)a.level_task0[l] + warp; t < t1; t += kGWarps) {
                const uint4 d = a.tasks[(size_t)t * RPT + slotr];  // row, off4, len4, task max len4
                uint4 acc = make_uint4(kInf16x2, kInf16x2, kInf16x2, kInf16x2);
                // eight entries (two loads of four) per pass, so eight row
                // loads are in flight per lane
                const uint4 pad4 = make_uint4(kGPad, kGPad, kGPad, kGPad);
                for (uint32_t e4 = 0; e4 < d.w; e4 += 2) {
                    const uint4 ea = e4 < d.z ? a.ents[mp_ix(d.y + e4, a.nents4, a.status)] : pad4;
                    const uint4 eb = e4 + 1 < d.z ? a.ents[mp_ix(d.y + e4 + 1, a.nents4, a.status)] : pad4;
                    const uint32_t e[8] = {ea.x, ea.y, ea.z, ea.w, eb.x, eb.y, eb.z, eb.w};
                    uint4 v[8];
                    uint32_t zz[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) gload(e[j], X, R, ldb, col, v[j], zz[j], N, a.status);
#pragma unroll
                    for (int j = 0; j < 8; ++j) gmin(acc, v[j], zz[j]);
                }
                if (d.x == 0xFFFFFFFFu) continue;
                const int64_t qr = mp_ix((int64_t)d.x, N, a.status);
                *reinterpret_cast<uint4 *>(R + qr * ldb + col) = acc;
                if (a.user_out)
                    store_row8(a.user_out + (kChain ? (size_t)(k - a.out_k0) * a.slot : 0) +
                                   (int64_t)mp_ix((int64_t)a.caller[qr], N, a.status) * N + a.col_base + col,
                               acc, N - a.col_base - col);
            }
            __syncthreads();  // this level's rows are read by the later levels
        }
        if (a.gdiag && warp < (W + 31) / 32) {
            int32_t v = (int32_t)kInf16;
            if (threadIdx.x < W && drow != 0xFFFFFFFFu)
                v = (int32_t)R[(int64_t)drow * ldb + cb + threadIdx.x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
            if (lane == 0 && v < (int32_t)kInf16) atomicMin(kChain ? a.gdiag + (k - a.out_k0) : a.gdiag, v);
        }
        if (kChain) {
            // the result is the next step's X; its old X becomes the next R
            // (every read of it in this step is before the last barrier)
            const uint16_t *nx = R;
            R = const_cast<uint16_t *>(X);
            X = nx;
        }
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace

int circuit_cover_structured(int n, const std::vector<uint32_t> &words, const std::vector<int32_t> &canon,
                             const HostCsr &csr, int lambda, CircuitCover *out) {
    const int64_t N = csr.N;
    if ((int64_t)words.size() != N || (int64_t)canon.size() != N)
        return set_error(MP_EINVAL, "structured cover: %lld words for %lld rows", (long long)words.size(),
                         (long long)N);
    if (N >= (int64_t)kGRow) return set_error(MP_EINVAL, "N = %lld too large for a circuit", (long long)N);
    CircuitCover &C = *out;
    C = CircuitCover();
    C.N = N;
    // internal row of every word, and the zero letters of every internal row
    // (bit j for letter j + 1, as in the word masks)
    std::vector<int32_t> inv((size_t)N);
    for (int64_t i = 0; i < N; ++i) inv[(size_t)canon[(size_t)i]] = (int32_t)i;
    auto letter = [&](uint32_t w, int j) { return (w >> (2 * (n - 1 - j))) & 3u; };
    std::vector<uint32_t> zm((size_t)N, 0);
    for (int64_t i = 0; i < N; ++i) {
        const uint32_t w = words[(size_t)canon[(size_t)i]];
        for (int j = 0; j < n; ++j)
            if (letter(w, j) == 0) zm[(size_t)i] |= 1u << j;
    }
    auto row_of = [&](uint32_t w) -> int64_t {  // internal row of a packed word, or -1
        auto it = std::lower_bound(words.begin(), words.end(), w);
        return (it != words.end() && *it == w) ? inv[(size_t)(it - words.begin())] : -1;
    };
    std::vector<int64_t> sz((size_t)N);
    for (int64_t q = 0; q < N; ++q) sz[(size_t)q] = csr.row_ptr[q + 1] - csr.row_ptr[q];
    std::vector<int64_t> order((size_t)N);
    for (int64_t q = 0; q < N; ++q) order[(size_t)q] = q;
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t x, int64_t y) { return sz[(size_t)x] < sz[(size_t)y]; });
    C.lists.assign((size_t)N, {});
    C.level.assign((size_t)N, 0);
    std::vector<int32_t> U, U2;
    struct Cand {
        int64_t row;
        uint32_t S;
    };
    std::vector<Cand> cand;
    std::vector<int> cnt1(16), cnt2(256);
    for (int64_t t = 0; t < N; ++t) {
        const int64_t q = order[(size_t)t];
        const uint32_t w = words[(size_t)canon[(size_t)q]];
        // candidates: one or two of q's 0/1 letters turned into 2, a correct word
        cand.clear();
        uint32_t allowed = 0;
        for (int j = 0; j < n; ++j) {
            if (letter(w, j) == 2) continue;
            const uint32_t wj = (w & ~(3u << (2 * (n - 1 - j)))) | (2u << (2 * (n - 1 - j)));
            const int64_t r = row_of(wj);
            if (r >= 0 && sz[(size_t)r] >= 2) cand.push_back({r, 1u << j});
            for (int j2 = j + 1; j2 < n; ++j2) {
                if (letter(w, j2) == 2) continue;
                const uint32_t wjj = (wj & ~(3u << (2 * (n - 1 - j2)))) | (2u << (2 * (n - 1 - j2)));
                const int64_t r2 = row_of(wjj);
                if (r2 >= 0 && sz[(size_t)r2] >= 2) cand.push_back({r2, (1u << j) | (1u << j2)});
            }
        }
        for (const Cand &c : cand) allowed |= c.S;
        U.assign(csr.col.begin() + csr.row_ptr[q], csr.col.begin() + csr.row_ptr[q + 1]);
        std::vector<uint32_t> &li = C.lists[(size_t)q];
        int lv = 0;
        while (!cand.empty() && !U.empty()) {
            // arcs still uncovered with a 0 at each letter, and at each pair
            std::fill(cnt1.begin(), cnt1.end(), 0);
            std::fill(cnt2.begin(), cnt2.end(), 0);
            for (int32_t p : U) {
                const uint32_t m = zm[(size_t)p] & allowed;
                for (uint32_t b = m; b; b &= b - 1) {
                    const int j = __builtin_ctz(b);
                    ++cnt1[(size_t)j];
                    for (uint32_t b2 = b & (b - 1); b2; b2 &= b2 - 1) ++cnt2[(size_t)(j * 16 + __builtin_ctz(b2))];
                }
            }
            int64_t best = -1, bs = 1;
            size_t bi = 0;
            for (size_t k = 0; k < cand.size(); ++k) {
                const uint32_t S = cand[k].S;
                const int j = __builtin_ctz(S);
                const int64_t g = (S & (S - 1)) ? cnt2[(size_t)(j * 16 + __builtin_ctz(S & (S - 1)))] : cnt1[(size_t)j];
                const int64_t added = std::max(0, C.level[(size_t)cand[k].row] + 1 - lv);
                const int64_t sc = g - (int64_t)lambda * added;
                if (g > 1 && sc > bs) {
                    bs = sc;
                    best = cand[k].row;
                    bi = k;
                }
            }
            if (best < 0) break;  // nothing left worth a cover: read the rest directly
            const uint32_t S = cand[bi].S;
            U2.clear();
            for (int32_t p : U)
                if ((zm[(size_t)p] & S) != S) U2.push_back(p);
            U.swap(U2);
            li.push_back((uint32_t)(N + best));
            lv = std::max(lv, C.level[(size_t)best] + 1);
            cand.erase(cand.begin() + (long)bi);
            ++C.cover_reads;
        }
        for (int32_t p : U) li.push_back((uint32_t)p);
        C.level[(size_t)q] = lv;
        C.reads += (int64_t)li.size();
        C.levels = std::max(C.levels, lv + 1);
    }
    return MP_OK;
}

int gcircuit_slice_host(const CircuitCover &cv, const std::vector<uint16_t> &z, int L, GCircuitHost *out) {
    if (L != 4 && L != 8 && L != 16 && L != 32) return set_error(MP_EINVAL, "lanes per row %d", L);
    const int64_t N = cv.N;
    const int RPT = 32 / L;
    GCircuitHost &G = *out;
    G = GCircuitHost();
    G.N = N;
    G.L = L;
    G.levels = cv.levels;
    G.reads = cv.reads;
    G.cover_reads = cv.cover_reads;
    G.level_task0.push_back(0);
    std::vector<std::vector<int64_t>> by_level((size_t)cv.levels);
    for (int64_t q = 0; q < N; ++q) by_level[(size_t)cv.level[(size_t)q]].push_back(q);
    for (int l = 0; l < cv.levels; ++l) {
        auto &rows = by_level[(size_t)l];
        std::stable_sort(rows.begin(), rows.end(), [&](int64_t x, int64_t y) {
            return cv.lists[(size_t)x].size() > cv.lists[(size_t)y].size();
        });
        for (size_t r0 = 0; r0 < rows.size(); r0 += (size_t)RPT) {
            const size_t r1 = std::min(rows.size(), r0 + (size_t)RPT);
            const uint32_t tmax = (uint32_t)((cv.lists[(size_t)rows[r0]].size() + 3) / 4);
            for (int i = 0; i < RPT; ++i) {
                if (r0 + (size_t)i >= r1) {
                    G.tasks.push_back({0xFFFFFFFFu, 0u, 0u, tmax});
                    continue;
                }
                const int64_t q = rows[r0 + (size_t)i];
                const auto &li = cv.lists[(size_t)q];
                const uint32_t off4 = (uint32_t)(G.ents.size() / 4);
                for (uint32_t v : li) {
                    if (v >= (uint32_t)N) {
                        G.ents.push_back(kGCover | (v - (uint32_t)N));
                    } else {
                        if (z[(size_t)v] > 15) return set_error(MP_EINVAL, "label %u too large", z[(size_t)v]);
                        G.ents.push_back(v | ((uint32_t)z[(size_t)v] << 24));
                    }
                }
                while (G.ents.size() % 4) G.ents.push_back(kGPad);
                G.tasks.push_back({(uint32_t)q, off4, (uint32_t)((li.size() + 3) / 4), tmax});
            }
        }
        G.level_task0.push_back((uint32_t)(G.tasks.size() / (size_t)RPT));
    }
    if (G.ents.empty())
        for (int i = 0; i < 4; ++i) G.ents.push_back(kGPad);
    if (G.ents.size() / 4 > 0xFFFFFFFFull) return set_error(MP_EINVAL, "circuit too large");
    return MP_OK;
}

int gcircuit_upload(const GCircuitHost &h, const std::vector<int32_t> &diagcol, const std::vector<int32_t> &caller,
                    PlanDev *d, cudaStream_t s) {
    GCircuitDev &g = d->gcircuit;
    g.ready = false;
    if ((int64_t)diagcol.size() != h.N || (int64_t)caller.size() != h.N || h.N != d->N)
        return set_error(MP_EINVAL, "circuit of the wrong size");
    const int W = 8 * h.L;
    if (d->ldb % W) return set_error(MP_EINVAL, "circuit chunk does not divide the buffer");
    std::vector<uint32_t> drow((size_t)d->ldb, 0xFFFFFFFFu);
    for (int64_t q = 0; q < h.N; ++q) {
        const int32_t dc = diagcol[(size_t)q];
        if (dc >= (int32_t)d->ldb || caller[(size_t)q] < 0)
            return set_error(MP_EINVAL, "circuit row fields out of range");
        if (dc >= 0) drow[(size_t)dc] = (uint32_t)q;
    }
    auto up = [&](DevBuf &buf, const void *src, size_t bytes) -> int {
        MP_TRY(buf.alloc(bytes ? bytes : 16, s, true));
        if (bytes) MP_CUDA_TRY(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, s));
        return MP_OK;
    };
    MP_TRY(up(g.level_task0, h.level_task0.data(), h.level_task0.size() * 4));
    MP_TRY(up(g.tasks, h.tasks.data(), h.tasks.size() * sizeof(uint4)));
    MP_TRY(up(g.ents, h.ents.data(), h.ents.size() * 4));
    MP_TRY(up(g.drow, drow.data(), drow.size() * 4));
    MP_TRY(up(g.caller, caller.data(), caller.size() * 4));
    MP_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors go out of scope
    g.L = h.L;
    g.levels = h.levels;
    g.reads = h.reads;
    g.cover_reads = h.cover_reads;
    g.bytes = h.level_task0.size() * 4 + h.tasks.size() * sizeof(uint4) + h.ents.size() * 4;
    g.ready = true;
    return MP_OK;
}

static int gcircuit_launch(const PlanDev &p, bool chain, const uint16_t *B0, uint16_t *B1, int k_max,
                           int16_t *user_out, size_t slot, int32_t *gdiag, cudaStream_t s, int out_k0,
                           int64_t col_base = 0, int64_t width = -1) {
    const GCircuitDev &g = p.gcircuit;
    if (!g.ready) return set_error(MP_EINVAL, "plan has no global circuit");
    if (p.narrow && user_out) return set_error(MP_EINVAL, "a narrow chain has no full powers to write");
    GArgs a;
    memset(&a, 0, sizeof(a));
    a.B0 = B0;
    a.B1 = B1;
    if (width < 0) width = p.ldb;
    const int W = 8 * g.L;
    if (col_base < 0 || col_base % W || width % W || col_base + width > p.ldb)
        return set_error(MP_EINVAL, "column block [%lld, +%lld) not on the circuit's chunks", (long long)col_base,
                         (long long)width);
    a.N = p.N;
    a.ldb = width;
    a.col_base = col_base;
    a.level_task0 = g.level_task0.as<uint32_t>();
    a.tasks = g.tasks.as<uint4>();
    a.ents = g.ents.as<uint4>();
    a.drow = g.drow.as<uint32_t>();
    a.caller = g.caller.as<int32_t>();
    a.levels = g.levels;
    a.k_max = k_max;
    a.out_k0 = out_k0;
    a.user_out = user_out;
    a.slot = slot;
    a.gdiag = gdiag;
    a.nents4 = (uint32_t)(g.ents.bytes / sizeof(uint4));
    MP_TRY(device_status_ptr(&a.status));
    const unsigned grid = (unsigned)(width / W);
    if (grid == 0) return MP_OK;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kGThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define MP_GLAUNCH(LL)                                                                       \
    MP_CUDA_TRY(chain ? cudaLaunchKernelEx(&cfg, gcircuit_kernel<LL, true>, a)               \
                      : cudaLaunchKernelEx(&cfg, gcircuit_kernel<LL, false>, a))
    switch (g.L) {
        case 4: MP_GLAUNCH(4); break;
        case 8: MP_GLAUNCH(8); break;
        case 16: MP_GLAUNCH(16); break;
        default: MP_GLAUNCH(32); break;
    }
#undef MP_GLAUNCH
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int gcircuit_step(const PlanDev &p, const uint16_t *Bin, uint16_t *Bout, int16_t *user_out, int32_t *gdiag,
                  cudaStream_t s) {
    return gcircuit_launch(p, false, Bin, Bout, 2, user_out, 0, gdiag, s, 1);
}

int gcircuit_chain(const PlanDev &p, uint16_t *B0, uint16_t *B1, int k_max, int16_t *powers, size_t slot,
                   int32_t *gdiag, cudaStream_t s, int out_k0) {
    if (k_max < 2) return MP_OK;
    if (powers && slot < (size_t)p.N * (size_t)p.N) return set_error(MP_EINVAL, "power slots too small");
    return gcircuit_launch(p, true, B0, B1, k_max, powers, slot, gdiag, s, out_k0);
}

int gcircuit_block_step(const PlanDev &p, const uint16_t *Bin, uint16_t *Bout, int64_t col_base, int64_t width,
                        int32_t *gdiag, cudaStream_t s) {
    return gcircuit_launch(p, false, Bin, Bout, 2, nullptr, 0, gdiag, s, 1, col_base, width);
}

int gcircuit_block_chain(const PlanDev &p, uint16_t *B0, uint16_t *B1, int k_max, int64_t col_base,
                         int64_t width, int32_t *gdiag, cudaStream_t s) {
    if (k_max < 2) return MP_OK;
    return gcircuit_launch(p, true, B0, B1, k_max, nullptr, 0, gdiag, s, 1, col_base, width);
}

int gcircuit_chunk(const PlanDev &p) { return p.gcircuit.ready ? 8 * p.gcircuit.L : 0; }

}  // namespace mp
