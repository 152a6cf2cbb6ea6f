// K1: dense exact (min,+) product Z = X (x) Y on the DPX integer pipe.
//
// Section 1 defines (X (x) Y)_ij = min_l (x_il + y_lj).  The entries are
// 16-bit (int16 storage, values in [0, 0x7FFF], INF = 0x7FFF) or 8-bit
// (values in [0, 255], INF = 255, widened to 16-bit lanes on chip).  Two
// output columns share one 32-bit register and every inner-loop step is a
// single __viaddmin_u16x2 (per halfword min(a + b, c)): the X value is
// stored twice in one word, the Y pair and the accumulator pair are two
// adjacent columns.  A lane sum is at most 0x7FFF + 0x7FFF = 0xFFFE, so the
// unsigned 16-bit add never wraps; the accumulator starts at INF and only
// decreases, so the result is min(INF, .) without a separate clamp.
//
// Tiling: a 128 x 128 output tile per CTA of 256 threads, K staged in
// steps of 32 through double-buffered shared memory, 8 x 8 outputs per
// thread (32 packed accumulators).  Blocks of 128 x 128 that are entirely
// INF in X or in Y (a precomputed occupancy mask per operand) cannot lower
// any minimum, so their K-range is skipped for the tile.
#include <algorithm>
#include <mutex>

#include "mp_internal.cuh"

namespace mp {

namespace {

constexpr int BM = 128, BN = 128, BK = 32, THREADS = 256;
constexpr int MASK_BLOCK = 128;

template <typename T> struct Elem;
template <> struct Elem<uint16_t> {
    static constexpr uint32_t inf = 0x7FFFu;
};
template <> struct Elem<uint8_t> {
    static constexpr uint32_t inf = 0xFFu;
};

__device__ __forceinline__ uint32_t dup16(uint32_t v) { return v | (v << 16); }

// Occupancy mask: mask[bi * nbc + bj] = 1 when the 128 x 128 block (bi, bj)
// holds at least one finite entry.
template <typename T>
__global__ void block_mask_kernel(const T *__restrict__ A, int64_t rows, int64_t cols,
                                  int64_t ld, uint8_t *__restrict__ mask, int64_t nbc) {
    int64_t bi = blockIdx.y, bj = blockIdx.x;
    int64_t r0 = bi * MASK_BLOCK, c0 = bj * MASK_BLOCK;
    int found = 0;
    for (int t = threadIdx.x; t < MASK_BLOCK * MASK_BLOCK && !found; t += blockDim.x) {
        int64_t r = r0 + t / MASK_BLOCK, c = c0 + t % MASK_BLOCK;
        if (r < rows && c < cols && (uint32_t)A[r * ld + c] < Elem<T>::inf) found = 1;
    }
    found = __syncthreads_or(found);
    if (threadIdx.x == 0) mask[bi * nbc + bj] = (uint8_t)(found ? 1 : 0);
}

template <typename T>
struct Stage {
    // register staging of one K-step: 16 X values and 16 Y values per thread
    uint32_t x[8];   // X[m][k0+kh .. +16] as 8 words of two 16-bit values
    uint32_t y[8];   // Y[k][n0+nc .. +16] widened to 16-bit, 8 words
};

template <typename T>
__device__ __forceinline__ void load_tile(const T *__restrict__ X, const T *__restrict__ Y,
                                          int64_t M, int64_t N, int64_t K, int64_t ldx,
                                          int64_t ldy, int64_t m0, int64_t n0, int64_t k0,
                                          bool vecx_ok, bool vecy_ok, Stage<T> &st) {
    const int t = threadIdx.x;
    const uint32_t inf = Elem<T>::inf;
    // X: row m = t/2, k half kh = (t&1)*16
    {
        int64_t m = m0 + (t >> 1), k = k0 + (t & 1) * 16;
        if (vecx_ok && m < M && k + 16 <= K) {
            const T *src = X + m * ldx + k;
            if (sizeof(T) == 2) {
                uint4 a = __ldg(reinterpret_cast<const uint4 *>(src));
                uint4 b = __ldg(reinterpret_cast<const uint4 *>(src) + 1);
                st.x[0] = a.x; st.x[1] = a.y; st.x[2] = a.z; st.x[3] = a.w;
                st.x[4] = b.x; st.x[5] = b.y; st.x[6] = b.z; st.x[7] = b.w;
            } else {
                uint4 a = __ldg(reinterpret_cast<const uint4 *>(src));
                uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    st.x[2 * j] = __byte_perm(w[j], 0, 0x4140);
                    st.x[2 * j + 1] = __byte_perm(w[j], 0, 0x4342);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                uint32_t lo = inf, hi = inf;
                if (m < M && k + 2 * j < K) lo = (uint32_t)X[m * ldx + k + 2 * j];
                if (m < M && k + 2 * j + 1 < K) hi = (uint32_t)X[m * ldx + k + 2 * j + 1];
                st.x[j] = lo | (hi << 16);
            }
        }
    }
    // Y: row k = t/8, columns nc = (t&7)*16
    {
        int64_t k = k0 + (t >> 3), n = n0 + (t & 7) * 16;
        if (vecy_ok && k < K && n + 16 <= N) {
            const T *src = Y + k * ldy + n;
            if (sizeof(T) == 2) {
                uint4 a = __ldg(reinterpret_cast<const uint4 *>(src));
                uint4 b = __ldg(reinterpret_cast<const uint4 *>(src) + 1);
                st.y[0] = a.x; st.y[1] = a.y; st.y[2] = a.z; st.y[3] = a.w;
                st.y[4] = b.x; st.y[5] = b.y; st.y[6] = b.z; st.y[7] = b.w;
            } else {
                uint4 a = __ldg(reinterpret_cast<const uint4 *>(src));
                uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    st.y[2 * j] = __byte_perm(w[j], 0, 0x4140);
                    st.y[2 * j + 1] = __byte_perm(w[j], 0, 0x4342);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                uint32_t lo = inf, hi = inf;
                if (k < K && n + 2 * j < N) lo = (uint32_t)Y[k * ldy + n + 2 * j];
                if (k < K && n + 2 * j + 1 < N) hi = (uint32_t)Y[k * ldy + n + 2 * j + 1];
                st.y[j] = lo | (hi << 16);
            }
        }
    }
}

template <typename T>
__device__ __forceinline__ void store_tile(const Stage<T> &st, uint32_t (*Xs)[BM],
                                           uint16_t (*Ys)[BN]) {
    const int t = threadIdx.x;
    const int m = t >> 1, kh = (t & 1) * 16;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        Xs[kh + 2 * j][m] = dup16(st.x[j] & 0xFFFFu);
        Xs[kh + 2 * j + 1][m] = dup16(st.x[j] >> 16);
    }
    const int k = t >> 3, nc = (t & 7) * 16;
    uint4 *dst = reinterpret_cast<uint4 *>(&Ys[k][nc]);
    dst[0] = make_uint4(st.y[0], st.y[1], st.y[2], st.y[3]);
    dst[1] = make_uint4(st.y[4], st.y[5], st.y[6], st.y[7]);
}

template <typename T>
struct TileArgs {
    const T *X;
    const T *Y;
    T *Z;
    int64_t M, N, K, ldx, ldy, ldz;
    const uint8_t *xmask, *ymask;  // occupancy masks, or NULL for "all active"
    int64_t kblocks, nblocks;
    int vecx, vecy, vecz;
    int32_t *gdiag;
};

// One 128 x 128 output tile (bi, bj) of Z = X (x) Y.  Ends with every thread
// past its last shared-memory read, so a persistent caller may start the
// next tile at once.
template <typename T>
__device__ __forceinline__ void gemm_tile(const TileArgs<T> &a, int64_t bi, int64_t bj,
                                          uint32_t (*Xs)[BK][BM], uint16_t (*Ys)[BK][BN]) {
    const T *__restrict__ X = a.X;
    const T *__restrict__ Y = a.Y;
    T *__restrict__ Z = a.Z;
    const int64_t M = a.M, N = a.N, K = a.K, ldx = a.ldx, ldy = a.ldy, ldz = a.ldz;
    const uint8_t *__restrict__ xmask = a.xmask;
    const uint8_t *__restrict__ ymask = a.ymask;
    const int64_t kblocks = a.kblocks, nblocks = a.nblocks;
    const int vecx = a.vecx, vecy = a.vecy, vecz = a.vecz;
    int32_t *__restrict__ gdiag = a.gdiag;
    const int64_t m0 = bi * BM, n0 = bj * BN;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const uint32_t inf2 = Elem<T>::inf * 0x10001u;

    uint32_t acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = inf2;

    const int64_t ktiles = (K + BK - 1) / BK;
    auto active = [&](int64_t kt) -> bool {
        if (!xmask) return true;
        int64_t kb = (kt * BK) / MASK_BLOCK;
        return xmask[bi * kblocks + kb] && ymask[kb * nblocks + bj];
    };
    auto next_active = [&](int64_t kt) -> int64_t {
        while (kt < ktiles && !active(kt)) ++kt;
        return kt;
    };

    Stage<T> st;
    int64_t kt = next_active(0);
    int buf = 0;
    if (kt < ktiles) {
        load_tile<T>(X, Y, M, N, K, ldx, ldy, m0, n0, kt * BK, vecx, vecy, st);
        store_tile<T>(st, Xs[0], Ys[0]);
    }
    __syncthreads();
    while (kt < ktiles) {
        int64_t kn = next_active(kt + 1);
        if (kn < ktiles) load_tile<T>(X, Y, M, N, K, ldx, ldy, m0, n0, kn * BK, vecx, vecy, st);
#pragma unroll 4
        for (int k = 0; k < BK; ++k) {
            uint4 xa = *reinterpret_cast<const uint4 *>(&Xs[buf][k][ty * 8]);
            uint4 xb = *reinterpret_cast<const uint4 *>(&Xs[buf][k][ty * 8 + 4]);
            uint4 yv = *reinterpret_cast<const uint4 *>(&Ys[buf][k][tx * 8]);
            const uint32_t xr[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
            const uint32_t yr[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = __viaddmin_u16x2(xr[r], yr[c], acc[r][c]);
        }
        if (kn < ktiles) store_tile<T>(st, Xs[buf ^ 1], Ys[buf ^ 1]);
        __syncthreads();
        buf ^= 1;
        kt = kn;
    }

    // epilogue
    int32_t dmin = 0x7FFFFFFF;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        int64_t m = m0 + ty * 8 + r;
        if (m >= M) continue;
        int64_t nb = n0 + tx * 8;
        T *zrow = Z + m * ldz;
        if (vecz && nb + 8 <= N) {
            if (sizeof(T) == 2) {
                *reinterpret_cast<uint4 *>(zrow + nb) = make_uint4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
            } else {
                uint32_t lo = __byte_perm(acc[r][0], acc[r][1], 0x6420);
                uint32_t hi = __byte_perm(acc[r][2], acc[r][3], 0x6420);
                *reinterpret_cast<uint2 *>(zrow + nb) = make_uint2(lo, hi);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (nb + 2 * c < N) zrow[nb + 2 * c] = (T)(acc[r][c] & 0xFFFFu);
                if (nb + 2 * c + 1 < N) zrow[nb + 2 * c + 1] = (T)(acc[r][c] >> 16);
            }
        }
        if (gdiag) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (nb + 2 * c == m) dmin = min(dmin, (int32_t)(acc[r][c] & 0xFFFFu));
                if (nb + 2 * c + 1 == m) dmin = min(dmin, (int32_t)(acc[r][c] >> 16));
            }
        }
    }
    if (gdiag && dmin != 0x7FFFFFFF) atomicMin(gdiag, dmin);
}

template <typename T>
__global__ void __launch_bounds__(THREADS) dense_minplus_kernel(TileArgs<T> a) {
    __shared__ __align__(16) uint32_t Xs[2][BK][BM];
    __shared__ __align__(16) uint16_t Ys[2][BK][BN];
    gemm_tile<T>(a, blockIdx.y, blockIdx.x, Xs, Ys);
}

template <typename T>
int run_dense(const T *X, const T *Y, T *Z, int64_t M, int64_t N, int64_t K, int64_t ldx,
              int64_t ldy, int64_t ldz, int32_t *gdiag, bool use_mask, cudaStream_t s) {
    const int64_t elems16 = 16 / (int64_t)sizeof(T);
    int vecx = ((uintptr_t)X % 16 == 0) && (ldx % elems16 == 0);
    int vecy = ((uintptr_t)Y % 16 == 0) && (ldy % elems16 == 0);
    // epilogue stores 8 outputs per row at a time: 16 B (int16) or 8 B (uint8)
    int vecz = ((uintptr_t)Z % 16 == 0) && (ldz % 8 == 0);
    const int64_t mb = (M + BM - 1) / BM, nb = (N + BN - 1) / BN;
    const int64_t kb = (K + MASK_BLOCK - 1) / MASK_BLOCK;
    DevBuf masks;
    const uint8_t *xm = nullptr, *ym = nullptr;
    if (use_mask && K > 0) {
        MP_TRY(masks.alloc((size_t)(mb * kb + kb * nb), s));
        uint8_t *xmw = masks.as<uint8_t>(), *ymw = xmw + mb * kb;
        block_mask_kernel<T><<<dim3((unsigned)kb, (unsigned)mb), 256, 0, s>>>(X, M, K, ldx, xmw, kb);
        block_mask_kernel<T><<<dim3((unsigned)nb, (unsigned)kb), 256, 0, s>>>(Y, K, N, ldy, ymw, nb);
        MP_CUDA_TRY(cudaGetLastError());
        xm = xmw;
        ym = ymw;
    }
    if (mb > 65535) return set_error(MP_EINVAL, "M = %lld too large for one launch", (long long)M);
    dim3 grid((unsigned)nb, (unsigned)mb);
    TileArgs<T> ta{X, Y, Z, M, N, K, ldx, ldy, ldz, xm, ym, kb, nb, vecx, vecy, vecz, gdiag};
    dense_minplus_kernel<T><<<grid, THREADS, 0, s>>>(ta);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

int dense_minplus(const void *X, const void *Y, void *Z, int64_t M, int64_t N, int64_t K,
                  int64_t ldx, int64_t ldy, int64_t ldz, int dtype, int32_t *gdiag,
                  cudaStream_t s) {
    if (M == 0 || N == 0) return MP_OK;
    if (dtype == MP_I16)
        return run_dense<uint16_t>((const uint16_t *)X, (const uint16_t *)Y, (uint16_t *)Z, M, N,
                                   K, ldx, ldy, ldz, gdiag, true, s);
    if (dtype == MP_U8)
        return run_dense<uint8_t>((const uint8_t *)X, (const uint8_t *)Y, (uint8_t *)Z, M, N, K,
                                  ldx, ldy, ldz, gdiag, true, s);
    return set_error(MP_EINVAL, "unknown dtype %d", dtype);
}

// ------------------------------------------------------------------ K5
// Many products of uneven sizes in one persistent launch.  The host lists
// every 128 x 128 output tile of every product, longest K first, and the
// CTAs (a full wave: 3 per SM) take tiles from an atomic counter until the
// list is exhausted.  The occupancy masks of all operands come from one
// preceding launch over a list of mask blocks.

namespace {

struct BatchProb {
    const void *X, *Y;
    void *Z;
    int64_t M, N, K, ldx, ldy, ldz;
    const uint8_t *xmask, *ymask;
    int64_t kblocks, nblocks;
    int32_t dtype, vecx, vecy, vecz;
};
struct BatchTile {
    int32_t prob, bi, bj, pad;
};
struct MaskJob {
    const void *A;
    int64_t rows, cols, ld, bi, bj, nbc;
    uint8_t *mask;
    int32_t dtype, pad;
};

__global__ void batched_mask_kernel(const MaskJob *__restrict__ jobs) {
    const MaskJob j = jobs[blockIdx.x];
    const int64_t r0 = j.bi * MASK_BLOCK, c0 = j.bj * MASK_BLOCK;
    const uint32_t inf = j.dtype == MP_I16 ? 0x7FFFu : 0xFFu;
    int found = 0;
    for (int t = threadIdx.x; t < MASK_BLOCK * MASK_BLOCK && !found; t += blockDim.x) {
        const int64_t r = r0 + t / MASK_BLOCK, c = c0 + t % MASK_BLOCK;
        if (r < j.rows && c < j.cols) {
            const uint32_t v = j.dtype == MP_I16
                                   ? (uint32_t)((const uint16_t *)j.A)[r * j.ld + c]
                                   : (uint32_t)((const uint8_t *)j.A)[r * j.ld + c];
            if (v < inf) found = 1;
        }
    }
    found = __syncthreads_or(found);
    if (threadIdx.x == 0) j.mask[j.bi * j.nbc + j.bj] = (uint8_t)(found ? 1 : 0);
}

__global__ void __launch_bounds__(THREADS, 2)
batched_minplus_kernel(const BatchProb *__restrict__ probs, const BatchTile *__restrict__ tiles,
                       int ntiles, int *counter) {
    __shared__ __align__(16) uint32_t Xs[2][BK][BM];
    __shared__ __align__(16) uint16_t Ys[2][BK][BN];
    __shared__ int next;
    while (true) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int t = next;
        __syncthreads();
        if (t >= ntiles) break;
        const BatchTile tl = tiles[t];
        const BatchProb &p = probs[tl.prob];
        if (p.dtype == MP_I16) {
            TileArgs<uint16_t> a{(const uint16_t *)p.X, (const uint16_t *)p.Y, (uint16_t *)p.Z,
                                 p.M, p.N, p.K, p.ldx, p.ldy, p.ldz, p.xmask, p.ymask,
                                 p.kblocks, p.nblocks, p.vecx, p.vecy, p.vecz, nullptr};
            gemm_tile<uint16_t>(a, tl.bi, tl.bj, Xs, Ys);
        } else {
            TileArgs<uint8_t> a{(const uint8_t *)p.X, (const uint8_t *)p.Y, (uint8_t *)p.Z,
                                p.M, p.N, p.K, p.ldx, p.ldy, p.ldz, p.xmask, p.ymask,
                                p.kblocks, p.nblocks, p.vecx, p.vecy, p.vecz, nullptr};
            gemm_tile<uint8_t>(a, tl.bi, tl.bj, Xs, Ys);
        }
    }
}

}  // namespace

int batched_run(const mp_problem *probs, int count, int mode, cudaStream_t s) {
    if (count == 0) return MP_OK;
    // validation (shared by both modes)
    for (int i = 0; i < count; ++i) {
        const mp_problem &p = probs[i];
        if (p.dtype != MP_I16 && p.dtype != MP_U8)
            return set_error(MP_EINVAL, "problem %d: dtype %d", i, p.dtype);
        if (p.M < 0 || p.N < 0 || p.K < 0)
            return set_error(MP_EINVAL, "problem %d: negative size", i);
        if (p.M == 0 || p.N == 0) continue;
        if (!p.Z || (p.K > 0 && (!p.X || !p.Y)))
            return set_error(MP_EINVAL, "problem %d: NULL pointer", i);
        if (p.ldx < std::max<int64_t>(p.K, 1) || p.ldy < p.N || p.ldz < p.N)
            return set_error(MP_EINVAL, "problem %d: leading dimension too small", i);
    }
    for (int i = 0; i < count; ++i) {
        const mp_problem &pi = probs[i];
        if (pi.M == 0 || pi.N == 0) continue;
        const size_t ei = pi.dtype == MP_I16 ? 2 : 1;
        const size_t zb = span_bytes(pi.M, pi.N, pi.ldz, ei);
        for (int j = 0; j < count; ++j) {
            const mp_problem &pj = probs[j];
            if (pj.M == 0 || pj.N == 0) continue;
            const size_t ej = pj.dtype == MP_I16 ? 2 : 1;
            if (ranges_overlap(pi.Z, zb, pj.X, span_bytes(pj.M, pj.K, pj.ldx, ej)) ||
                ranges_overlap(pi.Z, zb, pj.Y, span_bytes(pj.K, pj.N, pj.ldy, ej)) ||
                (i != j && ranges_overlap(pi.Z, zb, pj.Z, span_bytes(pj.M, pj.N, pj.ldz, ej))))
                return set_error(MP_EALIAS, "problem %d's output overlaps problem %d", i, j);
        }
    }
    if (mode == 1) {
        for (int i = 0; i < count; ++i) {
            const mp_problem &p = probs[i];
            MP_TRY(dense_minplus(p.X, p.Y, p.Z, p.M, p.N, p.K, p.ldx, p.ldy, p.ldz, p.dtype,
                                 nullptr, s));
        }
        return MP_OK;
    }
    // mode 0: masks for all operands in one launch, then one persistent launch
    std::vector<BatchProb> bp((size_t)count);
    std::vector<MaskJob> jobs;
    std::vector<BatchTile> tiles;
    std::vector<std::pair<int64_t, size_t>> order;  // (K, tile index) for longest-first
    size_t mask_bytes = 0;
    std::vector<size_t> xoff((size_t)count), yoff((size_t)count);
    for (int i = 0; i < count; ++i) {
        const mp_problem &p = probs[i];
        const int64_t mb = (p.M + BM - 1) / BM, nb = (p.N + BN - 1) / BN;
        const int64_t kb = (p.K + MASK_BLOCK - 1) / MASK_BLOCK;
        xoff[i] = mask_bytes;
        mask_bytes += (size_t)(mb * kb);
        yoff[i] = mask_bytes;
        mask_bytes += (size_t)(kb * nb);
    }
    DevBuf dmask, dprob, dtile, djob, dcnt;
    MP_TRY(dmask.alloc(std::max<size_t>(mask_bytes, 16), s));
    uint8_t *mbase = dmask.as<uint8_t>();
    for (int i = 0; i < count; ++i) {
        const mp_problem &p = probs[i];
        const int64_t e = p.dtype == MP_I16 ? 2 : 1;
        const int64_t mb = (p.M + BM - 1) / BM, nb = (p.N + BN - 1) / BN;
        const int64_t kb = (p.K + MASK_BLOCK - 1) / MASK_BLOCK;
        BatchProb &q = bp[i];
        q.X = p.X; q.Y = p.Y; q.Z = p.Z;
        q.M = p.M; q.N = p.N; q.K = p.K; q.ldx = p.ldx; q.ldy = p.ldy; q.ldz = p.ldz;
        q.kblocks = kb; q.nblocks = nb; q.dtype = p.dtype;
        q.vecx = ((uintptr_t)p.X % 16 == 0) && (p.ldx % (16 / e) == 0);
        q.vecy = ((uintptr_t)p.Y % 16 == 0) && (p.ldy % (16 / e) == 0);
        q.vecz = ((uintptr_t)p.Z % 16 == 0) && (p.ldz % 8 == 0);
        q.xmask = p.K > 0 ? mbase + xoff[i] : nullptr;
        q.ymask = p.K > 0 ? mbase + yoff[i] : nullptr;
        if (p.M == 0 || p.N == 0) continue;
        if (p.K > 0) {
            for (int64_t bi = 0; bi < mb; ++bi)
                for (int64_t bk = 0; bk < kb; ++bk)
                    jobs.push_back({p.X, p.M, p.K, p.ldx, bi, bk, kb, mbase + xoff[i], p.dtype, 0});
            for (int64_t bk = 0; bk < kb; ++bk)
                for (int64_t bj = 0; bj < nb; ++bj)
                    jobs.push_back({p.Y, p.K, p.N, p.ldy, bk, bj, nb, mbase + yoff[i], p.dtype, 0});
        }
        for (int64_t bi = 0; bi < mb; ++bi)
            for (int64_t bj = 0; bj < nb; ++bj) {
                order.push_back({p.K, tiles.size()});
                tiles.push_back({i, (int32_t)bi, (int32_t)bj, 0});
            }
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<int64_t, size_t> &a, const std::pair<int64_t, size_t> &b) {
                         return a.first > b.first;
                     });
    std::vector<BatchTile> sorted(tiles.size());
    for (size_t t = 0; t < order.size(); ++t) sorted[t] = tiles[order[t].second];
    MP_TRY(dprob.alloc(bp.size() * sizeof(BatchProb), s));
    MP_TRY(dtile.alloc(std::max<size_t>(sorted.size(), 1) * sizeof(BatchTile), s));
    MP_TRY(djob.alloc(std::max<size_t>(jobs.size(), 1) * sizeof(MaskJob), s));
    MP_TRY(dcnt.alloc(sizeof(int), s));
    MP_CUDA_TRY(cudaMemcpyAsync(dprob.p, bp.data(), bp.size() * sizeof(BatchProb),
                                cudaMemcpyHostToDevice, s));
    if (!sorted.empty())
        MP_CUDA_TRY(cudaMemcpyAsync(dtile.p, sorted.data(), sorted.size() * sizeof(BatchTile),
                                    cudaMemcpyHostToDevice, s));
    if (!jobs.empty())
        MP_CUDA_TRY(cudaMemcpyAsync(djob.p, jobs.data(), jobs.size() * sizeof(MaskJob),
                                    cudaMemcpyHostToDevice, s));
    MP_CUDA_TRY(cudaMemsetAsync(dcnt.p, 0, sizeof(int), s));
    for (size_t j0 = 0; j0 < jobs.size(); j0 += 1u << 30) {
        const size_t nj = std::min<size_t>(jobs.size() - j0, 1u << 30);
        batched_mask_kernel<<<(unsigned)nj, 256, 0, s>>>(djob.as<MaskJob>() + j0);
    }
    MP_CUDA_TRY(cudaGetLastError());
    if (!sorted.empty()) {
        DeviceInfo di;
        MP_TRY(device_info(&di));
        const int64_t grid = std::min<int64_t>((int64_t)sorted.size(), (int64_t)di.sms * 3);
        batched_minplus_kernel<<<(unsigned)grid, THREADS, 0, s>>>(
            dprob.as<BatchProb>(), dtile.as<BatchTile>(), (int)sorted.size(), dcnt.as<int>());
        MP_CUDA_TRY(cudaGetLastError());
    }
    return MP_OK;
}

// ------------------------------------------------- no-allocation variant
// mp_minplus_mul_noalloc: the same product for callers that cannot
// allocate device memory (see include/minplus.h).  The only scratch of the
// dense product -- the two occupancy masks -- lives in this fixed array,
// which every GPU that loads the library holds until the process exits.

namespace {

constexpr size_t kNoAllocMaskBytes = (size_t)1 << 20;  // 1 MiB of mask bytes
static __device__ __align__(256) uint8_t g_noalloc_masks[kNoAllocMaskBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[256] = {};

// Device address of g_noalloc_masks on the current device, looked up once
// per device with that device current.  In host code the array's name is
// only a host-side stand-in, never a device address.
int noalloc_scratch(uint8_t **out) {
    int dev = -1;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return set_error(MP_EINVAL, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_masks);
        if (e != cudaSuccess || !p)
            return set_error(MP_ECUDA, "cudaGetSymbolAddress(mask scratch) failed: %s",
                             cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<uint8_t *>(g_noalloc_addr[dev]);
    return MP_OK;
}

template <typename T>
int run_dense_noalloc(const T *X, const T *Y, T *Z, int64_t M, int64_t N, int64_t K,
                      int64_t ldx, int64_t ldy, int64_t ldz, cudaStream_t s) {
    const int64_t elems16 = 16 / (int64_t)sizeof(T);
    int vecx = ((uintptr_t)X % 16 == 0) && (ldx % elems16 == 0);
    int vecy = ((uintptr_t)Y % 16 == 0) && (ldy % elems16 == 0);
    int vecz = ((uintptr_t)Z % 16 == 0) && (ldz % 8 == 0);
    const int64_t mb = (M + BM - 1) / BM, nb = (N + BN - 1) / BN;
    const int64_t kb = (K + MASK_BLOCK - 1) / MASK_BLOCK;
    const uint8_t *xm = nullptr, *ym = nullptr;
    if (K > 0) {
        uint8_t *base = nullptr;
        MP_TRY(noalloc_scratch(&base));
        // every mask byte the product reads is written here first, so stale
        // contents of an earlier call never matter
        uint8_t *xmw = base, *ymw = base + mb * kb;
        block_mask_kernel<T><<<dim3((unsigned)kb, (unsigned)mb), 256, 0, s>>>(X, M, K, ldx, xmw, kb);
        block_mask_kernel<T><<<dim3((unsigned)nb, (unsigned)kb), 256, 0, s>>>(Y, K, N, ldy, ymw, nb);
        MP_CUDA_TRY(cudaGetLastError());
        xm = xmw;
        ym = ymw;
    }
    dim3 grid((unsigned)nb, (unsigned)mb);
    TileArgs<T> ta{X, Y, Z, M, N, K, ldx, ldy, ldz, xm, ym, kb, nb, vecx, vecy, vecz, nullptr};
    dense_minplus_kernel<T><<<grid, THREADS, 0, s>>>(ta);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

int dense_minplus_noalloc(const void *X, const void *Y, void *Z, int64_t M, int64_t N,
                          int64_t K, int64_t ldx, int64_t ldy, int64_t ldz, int dtype,
                          cudaStream_t s) {
    if (M == 0 || N == 0) return MP_OK;
    const int64_t mb = (M + BM - 1) / BM, nb = (N + BN - 1) / BN;
    const int64_t kb = (K + MASK_BLOCK - 1) / MASK_BLOCK;
    if (mb > 65535)
        return set_error(MP_EINVAL, "M = %lld too large for one launch", (long long)M);
    if ((double)(mb * kb + kb * nb) > (double)kNoAllocMaskBytes)
        return set_error(MP_EINVAL,
                         "problem needs %lld mask bytes; the fixed scratch holds %zu "
                         "(ceil(M/128)*ceil(K/128) + ceil(K/128)*ceil(N/128) must not exceed it)",
                         (long long)(mb * kb + kb * nb), kNoAllocMaskBytes);
    if (dtype == MP_I16)
        return run_dense_noalloc<uint16_t>((const uint16_t *)X, (const uint16_t *)Y,
                                           (uint16_t *)Z, M, N, K, ldx, ldy, ldz, s);
    if (dtype == MP_U8)
        return run_dense_noalloc<uint8_t>((const uint8_t *)X, (const uint8_t *)Y, (uint8_t *)Z,
                                          M, N, K, ldx, ldy, ldz, s);
    return set_error(MP_EINVAL, "unknown dtype %d", dtype);
}

}  // namespace mp
