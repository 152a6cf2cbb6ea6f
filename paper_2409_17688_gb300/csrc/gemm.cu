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
#include <map>
#include <memory>
#include <mutex>
#include <cstring>

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

// Occupancy mask: mask[bi * nbc + bj] = 1 when the 128 x 128 block (bi, bj)
// holds at least one finite entry.
// When dst is given the block is also copied there (leading dimension ldd):
// operands whose rows are not 16-byte aligned are repacked once so the
// product's tile loads can use 16-byte vectors.
template <typename T>
__global__ void block_mask_kernel(const T *__restrict__ A, int64_t rows, int64_t cols,
                                  int64_t ld, uint8_t *__restrict__ mask, int64_t nbc,
                                  T *__restrict__ dst, int64_t ldd) {
    int64_t bi = blockIdx.y, bj = blockIdx.x;
    int64_t r0 = bi * MASK_BLOCK, c0 = bj * MASK_BLOCK;
    int found = 0;
    for (int t = threadIdx.x; t < MASK_BLOCK * MASK_BLOCK && (dst || !found); t += blockDim.x) {
        int64_t r = r0 + t / MASK_BLOCK, c = c0 + t % MASK_BLOCK;
        if (r < rows && c < cols) {
            const T v = A[r * ld + c];
            if ((uint32_t)v < Elem<T>::inf) found = 1;
            if (dst) dst[r * ldd + c] = v;
        }
    }
    found = __syncthreads_or(found);
    if (threadIdx.x == 0) mask[bi * nbc + bj] = (uint8_t)(found ? 1 : 0);
}

// Tile shapes.  Both use 256 threads as a 16 x 16 grid, each thread owning
// TM rows x TN columns of the output tile (TN/2 packed accumulators per row).
template <int BM_, int BN_>
struct TileCfg {
    static constexpr int BM = BM_, BN = BN_;
    static constexpr int TM = BM_ / 16, TN = BN_ / 16;
    static constexpr int XSPLIT = THREADS / BM_;       // threads per X row
    static constexpr int XK = BK / XSPLIT;              // k values per thread (16 or 8)
    static constexpr int YP = BK * BN_ / 8 / THREADS;  // 8-column pieces of Y per thread
};
using Tile128 = TileCfg<128, 128>;
using Tile64 = TileCfg<64, 64>;

template <typename Cfg>
struct Stage {
    uint32_t x[Cfg::XK / 2];     // X[m][k0+kb .. +XK] as pairs of 16-bit values
    uint32_t y[Cfg::YP][4];      // Y[k][n0+nc .. +8] widened to 16-bit pairs
};

// Shared-memory tiles, sized for the larger shape and reused by the smaller.
struct TileSmem {
    uint32_t Xs[2][BK][BM];  // X^T, each value duplicated into both halves
    uint16_t Ys[2][BK][BN];
};

template <typename T>
__device__ __forceinline__ void widen8(const T *src, bool vec, uint32_t (&w)[4]) {
    if (sizeof(T) == 2) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(src));
        w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    } else {
        const uint2 a = __ldg(reinterpret_cast<const uint2 *>(src));
        w[0] = __byte_perm(a.x, 0, 0x4140);
        w[1] = __byte_perm(a.x, 0, 0x4342);
        w[2] = __byte_perm(a.y, 0, 0x4140);
        w[3] = __byte_perm(a.y, 0, 0x4342);
    }
}

template <typename T, typename Cfg>
__device__ __forceinline__ void load_tile(const T *__restrict__ X, const T *__restrict__ Y,
                                          int64_t M, int64_t N, int64_t K, int64_t ldx,
                                          int64_t ldy, int64_t m0, int64_t n0, int64_t k0,
                                          bool vecx_ok, bool vecy_ok, Stage<Cfg> &st) {
    const int t = threadIdx.x;
    const uint32_t inf = Elem<T>::inf;
    {
        const int64_t m = m0 + t / Cfg::XSPLIT, k = k0 + (t % Cfg::XSPLIT) * Cfg::XK;
#pragma unroll
        for (int pc = 0; pc < Cfg::XK / 8; ++pc) {
            const int64_t kk = k + 8 * pc;
            if (vecx_ok && m < M && kk + 8 <= K) {
                uint32_t w[4];
                widen8<T>(X + m * ldx + kk, true, w);
#pragma unroll
                for (int j = 0; j < 4; ++j) st.x[4 * pc + j] = w[j];
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint32_t lo = inf, hi = inf;
                    if (m < M && kk + 2 * j < K) lo = (uint32_t)X[m * ldx + kk + 2 * j];
                    if (m < M && kk + 2 * j + 1 < K) hi = (uint32_t)X[m * ldx + kk + 2 * j + 1];
                    st.x[4 * pc + j] = lo | (hi << 16);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < Cfg::YP; ++i) {
        const int pc = t + i * THREADS;
        const int64_t k = k0 + pc / (Cfg::BN / 8), n = n0 + (pc % (Cfg::BN / 8)) * 8;
        if (vecy_ok && k < K && n + 8 <= N) {
            widen8<T>(Y + k * ldy + n, true, st.y[i]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t lo = inf, hi = inf;
                if (k < K && n + 2 * j < N) lo = (uint32_t)Y[k * ldy + n + 2 * j];
                if (k < K && n + 2 * j + 1 < N) hi = (uint32_t)Y[k * ldy + n + 2 * j + 1];
                st.y[i][j] = lo | (hi << 16);
            }
        }
    }
}

template <typename Cfg>
__device__ __forceinline__ void store_tile(const Stage<Cfg> &st, TileSmem &sm, int buf) {
    const int t = threadIdx.x;
    const int m = t / Cfg::XSPLIT, kb = (t % Cfg::XSPLIT) * Cfg::XK;
    uint32_t *xs = &sm.Xs[buf][0][0];
#pragma unroll
    for (int j = 0; j < Cfg::XK / 2; ++j) {
        // each 16-bit value in both halves of a word (one byte permute)
        xs[(kb + 2 * j) * Cfg::BM + m] = __byte_perm(st.x[j], 0, 0x1010);
        xs[(kb + 2 * j + 1) * Cfg::BM + m] = __byte_perm(st.x[j], 0, 0x3232);
    }
    uint16_t *ys = &sm.Ys[buf][0][0];
#pragma unroll
    for (int i = 0; i < Cfg::YP; ++i) {
        const int pc = t + i * THREADS;
        const int k = pc / (Cfg::BN / 8), nc = (pc % (Cfg::BN / 8)) * 8;
        *reinterpret_cast<uint4 *>(ys + k * Cfg::BN + nc) =
            make_uint4(st.y[i][0], st.y[i][1], st.y[i][2], st.y[i][3]);
    }
}

template <typename T>
struct TileArgs {
    const T *X;
    const T *Y;
    T *Z;
    int64_t M, N, K, ldx, ldy, ldz;
    const uint8_t *xmask, *ymask;  // occupancy masks (128-blocks), or NULL for "all active"
    int64_t kblocks, nblocks;      // mask grid: K and N in 128-blocks
    int vecx, vecy, vecz;
    int32_t *gdiag;
};

// One output tile (bi, bj) of Z = X (x) Y in shape Cfg.  Ends with every
// thread past its last shared-memory read, so a persistent caller may start
// the next tile at once.
template <typename T, typename Cfg>
__device__ __forceinline__ void gemm_tile(const TileArgs<T> &a, int64_t bi, int64_t bj,
                                          TileSmem &sm) {
    constexpr int TM = Cfg::TM, TW = Cfg::TN / 2;
    const int64_t m0 = bi * Cfg::BM, n0 = bj * Cfg::BN;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const uint32_t inf2 = Elem<T>::inf * 0x10001u;
    const int64_t mb = m0 / MASK_BLOCK, nbk = n0 / MASK_BLOCK;

    uint32_t acc[TM][TW];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TW; ++c) acc[r][c] = inf2;

    const int64_t ktiles = (a.K + BK - 1) / BK;
    auto active = [&](int64_t kt) -> bool {
        if (!a.xmask) return true;
        const int64_t kb = (kt * BK) / MASK_BLOCK;
        return a.xmask[mb * a.kblocks + kb] && a.ymask[kb * a.nblocks + nbk];
    };
    auto next_active = [&](int64_t kt) -> int64_t {
        while (kt < ktiles && !active(kt)) ++kt;
        return kt;
    };

    Stage<Cfg> st;
    int64_t kt = next_active(0);
    int buf = 0;
    if (kt < ktiles) {
        load_tile<T, Cfg>(a.X, a.Y, a.M, a.N, a.K, a.ldx, a.ldy, m0, n0, kt * BK, a.vecx, a.vecy, st);
        store_tile<Cfg>(st, sm, 0);
    }
    __syncthreads();
    while (kt < ktiles) {
        const int64_t kn = next_active(kt + 1);
        if (kn < ktiles)
            load_tile<T, Cfg>(a.X, a.Y, a.M, a.N, a.K, a.ldx, a.ldy, m0, n0, kn * BK, a.vecx, a.vecy, st);
        const uint32_t *xs = &sm.Xs[buf][0][0];
        const uint16_t *ys = &sm.Ys[buf][0][0];
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            uint32_t xr[TM], yr[TW];
#pragma unroll
            for (int r = 0; r < TM; r += 4) {
                const uint4 v = *reinterpret_cast<const uint4 *>(xs + k * Cfg::BM + ty * TM + r);
                xr[r] = v.x; xr[r + 1] = v.y; xr[r + 2] = v.z; xr[r + 3] = v.w;
            }
            if (TW == 4) {
                const uint4 v = *reinterpret_cast<const uint4 *>(ys + k * Cfg::BN + tx * Cfg::TN);
                yr[0] = v.x; yr[1] = v.y; yr[2 % TW] = v.z; yr[3 % TW] = v.w;
            } else {
                const uint2 v = *reinterpret_cast<const uint2 *>(ys + k * Cfg::BN + tx * Cfg::TN);
                yr[0] = v.x; yr[1 % TW] = v.y;
            }
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int c = 0; c < TW; ++c) acc[r][c] = __viaddmin_u16x2(xr[r], yr[c], acc[r][c]);
        }
        if (kn < ktiles) store_tile<Cfg>(st, sm, buf ^ 1);
        __syncthreads();
        buf ^= 1;
        kt = kn;
    }

    // epilogue
    int32_t dmin = 0x7FFFFFFF;
#pragma unroll
    for (int r = 0; r < TM; ++r) {
        const int64_t m = m0 + ty * TM + r;
        if (m >= a.M) continue;
        const int64_t nb = n0 + tx * Cfg::TN;
        T *zrow = a.Z + m * a.ldz;
        if (a.vecz && nb + Cfg::TN <= a.N) {
            if (sizeof(T) == 2) {
                if (TW == 4)
                    *reinterpret_cast<uint4 *>(zrow + nb) = make_uint4(acc[r][0], acc[r][1 % TW], acc[r][2 % TW], acc[r][3 % TW]);
                else
                    *reinterpret_cast<uint2 *>(zrow + nb) = make_uint2(acc[r][0], acc[r][1 % TW]);
            } else {
                const uint32_t lo = __byte_perm(acc[r][0], acc[r][1 % TW], 0x6420);
                if (TW == 4) {
                    const uint32_t hi = __byte_perm(acc[r][2 % TW], acc[r][3 % TW], 0x6420);
                    *reinterpret_cast<uint2 *>(zrow + nb) = make_uint2(lo, hi);
                } else {
                    *reinterpret_cast<uint32_t *>(zrow + nb) = lo;
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < TW; ++c) {
                if (nb + 2 * c < a.N) zrow[nb + 2 * c] = (T)(acc[r][c] & 0xFFFFu);
                if (nb + 2 * c + 1 < a.N) zrow[nb + 2 * c + 1] = (T)(acc[r][c] >> 16);
            }
        }
        if (a.gdiag) {
#pragma unroll
            for (int c = 0; c < TW; ++c) {
                if (nb + 2 * c == m) dmin = min(dmin, (int32_t)(acc[r][c] & 0xFFFFu));
                if (nb + 2 * c + 1 == m) dmin = min(dmin, (int32_t)(acc[r][c] >> 16));
            }
        }
    }
    if (a.gdiag && dmin != 0x7FFFFFFF) atomicMin(a.gdiag, dmin);
}

template <typename T, typename Cfg>
__global__ void __launch_bounds__(THREADS) dense_minplus_kernel(TileArgs<T> a) {
    __shared__ __align__(16) TileSmem sm;
    gemm_tile<T, Cfg>(a, blockIdx.y, blockIdx.x, sm);
}

// ------------------------------------------------------- tile-shape tuning
// Size classes by min(M, N): [0,128) [128,256) [256,512) [512,1024)
// [1024,2048) [2048,inf).  The table holds the tile shape (0: 128x128,
// 1: 64x64) per element type and class, per device; mp_autotune measures it.
constexpr int kClasses = 6;
struct TuneTable {
    int32_t cfg[2][kClasses];
};
std::mutex g_tune_mu;
std::map<int, TuneTable> g_tune;

int size_class(int64_t M, int64_t N) {
    const int64_t s = std::min(M, N);
    int c = 0;
    for (int64_t lim = 128; c < kClasses - 1 && s >= lim; lim *= 2) ++c;
    return c;
}

TuneTable default_table() {
    TuneTable t;
    for (int d = 0; d < 2; ++d)
        for (int c = 0; c < kClasses; ++c) t.cfg[d][c] = c < 2 ? 1 : 0;
    return t;
}

int current_table(TuneTable *out) {
    int dev = -1;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(dev);
    *out = it == g_tune.end() ? default_table() : it->second;
    return MP_OK;
}

int choose_cfg(int dtype, int64_t M, int64_t N, int *cfg) {
    TuneTable t;
    MP_TRY(current_table(&t));
    *cfg = t.cfg[dtype == MP_U8 ? 1 : 0][size_class(M, N)];
    return MP_OK;
}

// Rows start on 8-element boundaries (what the 8-element vector loads of a
// tile need).
template <typename T>
bool rows_aligned(const T *A, int64_t ld) {
    return (uintptr_t)A % (8 * sizeof(T)) == 0 && ld % 8 == 0;
}

template <typename T>
TileArgs<T> make_args(const T *X, const T *Y, T *Z, int64_t M, int64_t N, int64_t K, int64_t ldx,
                      int64_t ldy, int64_t ldz, const uint8_t *xm, const uint8_t *ym,
                      int32_t *gdiag) {
    const int64_t nb128 = (N + MASK_BLOCK - 1) / MASK_BLOCK;
    const int64_t kb = (K + MASK_BLOCK - 1) / MASK_BLOCK;
    TileArgs<T> ta;
    ta.X = X; ta.Y = Y; ta.Z = Z;
    ta.M = M; ta.N = N; ta.K = K; ta.ldx = ldx; ta.ldy = ldy; ta.ldz = ldz;
    ta.xmask = xm; ta.ymask = ym; ta.kblocks = kb; ta.nblocks = nb128;
    // vector loads of 8 elements need 8-element-aligned rows
    ta.vecx = rows_aligned(X, ldx);
    ta.vecy = rows_aligned(Y, ldy);
    // the epilogue stores up to 8 outputs of a row at once
    ta.vecz = ((uintptr_t)Z % 16 == 0) && (ldz % 8 == 0);
    ta.gdiag = gdiag;
    return ta;
}

template <typename T>
int launch_product(const TileArgs<T> &ta, int cfg, cudaStream_t s) {
    const int bm = cfg == 1 ? 64 : 128;
    const int64_t mb = (ta.M + bm - 1) / bm, nb = (ta.N + bm - 1) / bm;
    if (mb > 65535) return set_error(MP_EINVAL, "M = %lld too large for one launch", (long long)ta.M);
    dim3 grid((unsigned)nb, (unsigned)mb);
    if (cfg == 1) dense_minplus_kernel<T, Tile64><<<grid, THREADS, 0, s>>>(ta);
    else dense_minplus_kernel<T, Tile128><<<grid, THREADS, 0, s>>>(ta);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

template <typename T>
int run_dense(const T *X, const T *Y, T *Z, int64_t M, int64_t N, int64_t K, int64_t ldx,
              int64_t ldy, int64_t ldz, int32_t *gdiag, int cfg, cudaStream_t s) {
    const int64_t mb = (M + MASK_BLOCK - 1) / MASK_BLOCK, nb = (N + MASK_BLOCK - 1) / MASK_BLOCK;
    const int64_t kb = (K + MASK_BLOCK - 1) / MASK_BLOCK;
    DevBuf masks, xpad, ypad;
    const uint8_t *xm = nullptr, *ym = nullptr;
    if (K > 0) {
        MP_TRY(masks.alloc((size_t)(mb * kb + kb * nb), s));
        uint8_t *xmw = masks.as<uint8_t>(), *ymw = xmw + mb * kb;
        // operands with rows off the 16-byte grid are repacked while masked
        T *xd = nullptr, *yd = nullptr;
        const int64_t ldxp = (K + 7) / 8 * 8, ldyp = (N + 7) / 8 * 8;
        if (!rows_aligned(X, ldx)) {
            MP_TRY(xpad.alloc((size_t)M * (size_t)ldxp * sizeof(T), s));
            xd = xpad.as<T>();
        }
        if (!rows_aligned(Y, ldy)) {
            MP_TRY(ypad.alloc((size_t)K * (size_t)ldyp * sizeof(T), s));
            yd = ypad.as<T>();
        }
        block_mask_kernel<T><<<dim3((unsigned)kb, (unsigned)mb), 256, 0, s>>>(X, M, K, ldx, xmw, kb,
                                                                           xd, ldxp);
        block_mask_kernel<T><<<dim3((unsigned)nb, (unsigned)kb), 256, 0, s>>>(Y, K, N, ldy, ymw, nb,
                                                                           yd, ldyp);
        MP_CUDA_TRY(cudaGetLastError());
        xm = xmw;
        ym = ymw;
        if (xd) {
            X = xd;
            ldx = ldxp;
        }
        if (yd) {
            Y = yd;
            ldy = ldyp;
        }
    }
    return launch_product<T>(make_args<T>(X, Y, Z, M, N, K, ldx, ldy, ldz, xm, ym, gdiag), cfg, s);
}

}  // namespace

int dense_minplus(const void *X, const void *Y, void *Z, int64_t M, int64_t N, int64_t K,
                  int64_t ldx, int64_t ldy, int64_t ldz, int dtype, int32_t *gdiag,
                  cudaStream_t s) {
    if (M == 0 || N == 0) return MP_OK;
    int cfg = 0;
    MP_TRY(choose_cfg(dtype, M, N, &cfg));
    if (dtype == MP_I16)
        return run_dense<uint16_t>((const uint16_t *)X, (const uint16_t *)Y, (uint16_t *)Z, M, N,
                                   K, ldx, ldy, ldz, gdiag, cfg, s);
    if (dtype == MP_U8)
        return run_dense<uint8_t>((const uint8_t *)X, (const uint8_t *)Y, (uint8_t *)Z, M, N, K,
                                  ldx, ldy, ldz, gdiag, cfg, s);
    return set_error(MP_EINVAL, "unknown dtype %d", dtype);
}

// ------------------------------------------------------------------ K5
// Many products of uneven sizes.  mp_batch_prepare lists every output tile
// of every product (in the tile shape the tuning table gives its size
// class), most expensive first, uploads that list with the problem
// descriptors and the list of occupancy-mask blocks, and owns the mask
// buffer.  mp_batch_run then only launches kernels (so it can be captured
// in a CUDA graph): mode 0 one mask launch and one persistent launch whose
// CTAs (a full wave) take tiles from an atomic counter; mode 1 a mask launch
// and a product launch per problem, the plain form.

namespace {

struct BatchProb {
    const void *X, *Y;
    void *Z;
    int64_t M, N, K, ldx, ldy, ldz;
    const uint8_t *xmask, *ymask;
    int64_t kblocks, nblocks;
    int32_t dtype, vecx, vecy, vecz;
    int32_t cfg, job0, job1, pad;
};
struct BatchTile {
    int32_t prob, bi, bj, cfg;
};
struct MaskJob {
    const void *A;
    int64_t rows, cols, ld, bi, bj, nbc;
    uint8_t *mask;
    void *dst;    // repacked copy of the block (leading dimension ldd), or NULL
    int64_t ldd;
    int32_t dtype, pad;
};

__global__ void batched_mask_kernel(const MaskJob *__restrict__ jobs) {
    const MaskJob j = jobs[blockIdx.x];
    const int64_t r0 = j.bi * MASK_BLOCK, c0 = j.bj * MASK_BLOCK;
    const bool i16 = j.dtype == MP_I16;
    const uint32_t inf = i16 ? 0x7FFFu : 0xFFu;
    int found = 0;
    for (int t = threadIdx.x; t < MASK_BLOCK * MASK_BLOCK && (j.dst || !found); t += blockDim.x) {
        const int64_t r = r0 + t / MASK_BLOCK, c = c0 + t % MASK_BLOCK;
        if (r < j.rows && c < j.cols) {
            const uint32_t v = i16 ? (uint32_t)((const uint16_t *)j.A)[r * j.ld + c]
                                   : (uint32_t)((const uint8_t *)j.A)[r * j.ld + c];
            if (v < inf) found = 1;
            if (j.dst) {
                if (i16) ((uint16_t *)j.dst)[r * j.ldd + c] = (uint16_t)v;
                else ((uint8_t *)j.dst)[r * j.ldd + c] = (uint8_t)v;
            }
        }
    }
    found = __syncthreads_or(found);
    if (threadIdx.x == 0) j.mask[j.bi * j.nbc + j.bj] = (uint8_t)(found ? 1 : 0);
}

template <typename T>
__device__ __forceinline__ TileArgs<T> prob_args(const BatchProb &p) {
    TileArgs<T> a;
    a.X = (const T *)p.X; a.Y = (const T *)p.Y; a.Z = (T *)p.Z;
    a.M = p.M; a.N = p.N; a.K = p.K; a.ldx = p.ldx; a.ldy = p.ldy; a.ldz = p.ldz;
    a.xmask = p.xmask; a.ymask = p.ymask; a.kblocks = p.kblocks; a.nblocks = p.nblocks;
    a.vecx = p.vecx; a.vecy = p.vecy; a.vecz = p.vecz;
    a.gdiag = nullptr;
    return a;
}

template <typename T>
__global__ void __launch_bounds__(THREADS, 2)
batched_minplus_kernel(const BatchProb *__restrict__ probs, const BatchTile *__restrict__ tiles,
                       int ntiles, int *counter) {
    __shared__ __align__(16) TileSmem sm;
    __shared__ int next;
    while (true) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        const int t = next;
        __syncthreads();
        if (t >= ntiles) break;
        const BatchTile tl = tiles[t];
        const TileArgs<T> a = prob_args<T>(probs[tl.prob]);
        if (tl.cfg == 1) gemm_tile<T, Tile64>(a, tl.bi, tl.bj, sm);
        else gemm_tile<T, Tile128>(a, tl.bi, tl.bj, sm);
    }
}

}  // namespace

}  // namespace mp

struct mp_batch {
    int count = 0, ntiles = 0, njobs = 0, grid = 0;
    int ntiles16 = 0;  // the int16 tiles come first in the list, then the uint8 ones
    std::vector<mp::BatchProb> host_probs;
    mp::DevBuf masks, probs, tiles, jobs, counter;
    mp::DevBuf pads;   // repacked copies of operands whose rows are off the 8-element grid
};

namespace mp {

int batch_prepare(const mp_problem *probs, int count, mp_batch **out) {
    if (count < 0 || (count > 0 && !probs)) return set_error(MP_EINVAL, "bad problem list");
    for (int i = 0; i < count; ++i) {
        const mp_problem &p = probs[i];
        if (p.dtype != MP_I16 && p.dtype != MP_U8)
            return set_error(MP_EINVAL, "problem %d: dtype %d", i, p.dtype);
        if (p.M < 0 || p.N < 0 || p.K < 0) return set_error(MP_EINVAL, "problem %d: negative size", i);
        if (p.M == 0 || p.N == 0) continue;
        if (!p.Z || (p.K > 0 && (!p.X || !p.Y)))
            return set_error(MP_EINVAL, "problem %d: NULL pointer", i);
        if (p.ldx < std::max<int64_t>(p.K, 1) || p.ldy < p.N || p.ldz < p.N)
            return set_error(MP_EINVAL, "problem %d: leading dimension too small", i);
        if ((p.M + 63) / 64 > 65535) return set_error(MP_EINVAL, "problem %d: M too large", i);
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
    TuneTable tune;
    MP_TRY(current_table(&tune));
    DeviceInfo di;
    MP_TRY(device_info(&di));
    auto b = std::make_unique<mp_batch>();
    b->count = count;
    b->host_probs.resize((size_t)count);
    std::vector<MaskJob> jobs;
    std::vector<std::pair<double, BatchTile>> order;
    size_t mask_bytes = 0;
    std::vector<size_t> xoff((size_t)count), yoff((size_t)count);
    for (int i = 0; i < count; ++i) {
        const mp_problem &p = probs[i];
        const int64_t mb = (p.M + MASK_BLOCK - 1) / MASK_BLOCK, nb = (p.N + MASK_BLOCK - 1) / MASK_BLOCK;
        const int64_t kb = (p.K + MASK_BLOCK - 1) / MASK_BLOCK;
        xoff[i] = mask_bytes;
        mask_bytes += (size_t)(mb * kb);
        yoff[i] = mask_bytes;
        mask_bytes += (size_t)(kb * nb);
    }
    MP_TRY(b->masks.alloc(std::max<size_t>(mask_bytes, 16), nullptr, true));
    uint8_t *mbase = b->masks.as<uint8_t>();
    // operands whose rows are not on the 8-element grid get a repacked copy
    // (written by the mask pass of every run) so their tiles load 16 bytes
    auto aligned8 = [](const void *A, int64_t ld, size_t e) {
        return (uintptr_t)A % (8 * e) == 0 && ld % 8 == 0;
    };
    std::vector<size_t> xpo((size_t)count, SIZE_MAX), ypo((size_t)count, SIZE_MAX);
    size_t pad_bytes = 0;
    for (int i = 0; i < count; ++i) {
        const mp_problem &p = probs[i];
        if (p.M == 0 || p.N == 0 || p.K == 0) continue;
        const size_t e = p.dtype == MP_I16 ? 2 : 1;
        if (!aligned8(p.X, p.ldx, e)) {
            xpo[i] = pad_bytes;
            pad_bytes += ((size_t)p.M * (size_t)((p.K + 7) / 8 * 8) * e + 255) / 256 * 256;
        }
        if (!aligned8(p.Y, p.ldy, e)) {
            ypo[i] = pad_bytes;
            pad_bytes += ((size_t)p.K * (size_t)((p.N + 7) / 8 * 8) * e + 255) / 256 * 256;
        }
    }
    if (pad_bytes) MP_TRY(b->pads.alloc(pad_bytes, nullptr, true));
    uint8_t *pbase = b->pads.as<uint8_t>();
    for (int i = 0; i < count; ++i) {
        const mp_problem &p = probs[i];
        const int64_t mb = (p.M + MASK_BLOCK - 1) / MASK_BLOCK, nb = (p.N + MASK_BLOCK - 1) / MASK_BLOCK;
        const int64_t kb = (p.K + MASK_BLOCK - 1) / MASK_BLOCK;
        const int cfg = tune.cfg[p.dtype == MP_U8 ? 1 : 0][size_class(p.M, p.N)];
        BatchProb &q = b->host_probs[i];
        const size_t e = p.dtype == MP_I16 ? 2 : 1;
        void *xd = xpo[i] != SIZE_MAX ? pbase + xpo[i] : nullptr;
        void *yd = ypo[i] != SIZE_MAX ? pbase + ypo[i] : nullptr;
        const int64_t ldxp = (p.K + 7) / 8 * 8, ldyp = (p.N + 7) / 8 * 8;
        q.X = xd ? xd : p.X; q.Y = yd ? yd : p.Y; q.Z = p.Z;
        q.M = p.M; q.N = p.N; q.K = p.K; q.ldz = p.ldz;
        q.ldx = xd ? ldxp : p.ldx;
        q.ldy = yd ? ldyp : p.ldy;
        q.kblocks = kb; q.nblocks = nb; q.dtype = p.dtype; q.cfg = cfg;
        q.vecx = aligned8(q.X, q.ldx, e);
        q.vecy = aligned8(q.Y, q.ldy, e);
        q.vecz = ((uintptr_t)p.Z % 16 == 0) && (p.ldz % 8 == 0);
        q.xmask = p.K > 0 ? mbase + xoff[i] : nullptr;
        q.ymask = p.K > 0 ? mbase + yoff[i] : nullptr;
        q.job0 = (int32_t)jobs.size();
        if (p.M > 0 && p.N > 0 && p.K > 0) {
            for (int64_t bi = 0; bi < mb; ++bi)
                for (int64_t bk = 0; bk < kb; ++bk)
                    jobs.push_back({p.X, p.M, p.K, p.ldx, bi, bk, kb, mbase + xoff[i], xd, ldxp, p.dtype, 0});
            for (int64_t bk = 0; bk < kb; ++bk)
                for (int64_t bj = 0; bj < nb; ++bj)
                    jobs.push_back({p.Y, p.K, p.N, p.ldy, bk, bj, nb, mbase + yoff[i], yd, ldyp, p.dtype, 0});
        }
        q.job1 = (int32_t)jobs.size();
        q.pad = 0;
        if (p.M == 0 || p.N == 0) continue;
        const int bm = cfg == 1 ? 64 : 128;
        const int64_t tm = (p.M + bm - 1) / bm, tn = (p.N + bm - 1) / bm;
        for (int64_t bi = 0; bi < tm; ++bi)
            for (int64_t bj = 0; bj < tn; ++bj)
                order.push_back({(double)p.K * bm * bm, {i, (int32_t)bi, (int32_t)bj, cfg}});
    }
    // int16 tiles first, then uint8 (one persistent launch per element
    // type); within each, the most expensive first
    auto is8 = [&](const BatchTile &t) { return probs[t.prob].dtype == MP_U8; };
    std::stable_sort(order.begin(), order.end(),
                     [&](const std::pair<double, BatchTile> &x, const std::pair<double, BatchTile> &y) {
                         if (is8(x.second) != is8(y.second)) return !is8(x.second);
                         return x.first > y.first;
                     });
    std::vector<BatchTile> tiles(order.size());
    int n16 = 0;
    for (size_t t = 0; t < order.size(); ++t) {
        tiles[t] = order[t].second;
        if (!is8(tiles[t])) ++n16;
    }
    b->ntiles16 = n16;
    b->ntiles = (int)tiles.size();
    b->njobs = (int)jobs.size();
    b->grid = (int)std::min<int64_t>((int64_t)tiles.size(), (int64_t)di.sms * 2);
    MP_TRY(b->probs.alloc(std::max<size_t>(b->host_probs.size(), 1) * sizeof(BatchProb), nullptr, true));
    MP_TRY(b->tiles.alloc(std::max<size_t>(tiles.size(), 1) * sizeof(BatchTile), nullptr, true));
    MP_TRY(b->jobs.alloc(std::max<size_t>(jobs.size(), 1) * sizeof(MaskJob), nullptr, true));
    MP_TRY(b->counter.alloc(2 * sizeof(int), nullptr, true));
    if (count)
        MP_CUDA_TRY(cudaMemcpy(b->probs.p, b->host_probs.data(), b->host_probs.size() * sizeof(BatchProb),
                               cudaMemcpyHostToDevice));
    if (!tiles.empty())
        MP_CUDA_TRY(cudaMemcpy(b->tiles.p, tiles.data(), tiles.size() * sizeof(BatchTile),
                               cudaMemcpyHostToDevice));
    if (!jobs.empty())
        MP_CUDA_TRY(cudaMemcpy(b->jobs.p, jobs.data(), jobs.size() * sizeof(MaskJob),
                               cudaMemcpyHostToDevice));
    *out = b.release();
    return MP_OK;
}

int batch_run(mp_batch *b, int mode, cudaStream_t s) {
    if (!b) return set_error(MP_EINVAL, "NULL batch");
    if (mode != 0 && mode != 1) return set_error(MP_EINVAL, "mode %d", mode);
    const MaskJob *jobs = b->jobs.as<MaskJob>();
    if (mode == 0) {
        for (int j0 = 0; j0 < b->njobs; j0 += 1 << 30) {
            const int nj = std::min(b->njobs - j0, 1 << 30);
            batched_mask_kernel<<<(unsigned)nj, 256, 0, s>>>(jobs + j0);
        }
        MP_CUDA_TRY(cudaGetLastError());
        if (b->ntiles > 0) {
            MP_CUDA_TRY(cudaMemsetAsync(b->counter.p, 0, 2 * sizeof(int), s));
            const int n16 = b->ntiles16, n8 = b->ntiles - b->ntiles16;
            if (n16 > 0)
                batched_minplus_kernel<uint16_t><<<(unsigned)std::min(b->grid, n16), THREADS, 0, s>>>(
                    b->probs.as<BatchProb>(), b->tiles.as<BatchTile>(), n16, b->counter.as<int>());
            if (n8 > 0)
                batched_minplus_kernel<uint8_t><<<(unsigned)std::min(b->grid, n8), THREADS, 0, s>>>(
                    b->probs.as<BatchProb>(), b->tiles.as<BatchTile>() + n16, n8,
                    b->counter.as<int>() + 1);
            MP_CUDA_TRY(cudaGetLastError());
        }
        return MP_OK;
    }
    for (int i = 0; i < b->count; ++i) {
        const BatchProb &p = b->host_probs[i];
        if (p.M == 0 || p.N == 0) continue;
        if (p.job1 > p.job0) batched_mask_kernel<<<(unsigned)(p.job1 - p.job0), 256, 0, s>>>(jobs + p.job0);
        MP_CUDA_TRY(cudaGetLastError());
        if (p.dtype == MP_I16) {
            TileArgs<uint16_t> ta = make_args<uint16_t>((const uint16_t *)p.X, (const uint16_t *)p.Y,
                                                        (uint16_t *)p.Z, p.M, p.N, p.K, p.ldx, p.ldy,
                                                        p.ldz, p.xmask, p.ymask, nullptr);
            MP_TRY(launch_product<uint16_t>(ta, p.cfg, s));
        } else {
            TileArgs<uint8_t> ta = make_args<uint8_t>((const uint8_t *)p.X, (const uint8_t *)p.Y,
                                                      (uint8_t *)p.Z, p.M, p.N, p.K, p.ldx, p.ldy,
                                                      p.ldz, p.xmask, p.ymask, nullptr);
            MP_TRY(launch_product<uint8_t>(ta, p.cfg, s));
        }
    }
    return MP_OK;
}

int batch_destroy(mp_batch *b) {
    delete b;
    return MP_OK;
}

int batched_run(const mp_problem *probs, int count, int mode, cudaStream_t s) {
    if (mode != 0 && mode != 1) return set_error(MP_EINVAL, "mode %d", mode);
    mp_batch *b = nullptr;
    MP_TRY(batch_prepare(probs, count, &b));
    int rc = batch_run(b, mode, s);
    // the descriptors must outlive the launches
    cudaError_t e = cudaStreamSynchronize(s);
    batch_destroy(b);
    if (rc != MP_OK) return rc;
    if (e != cudaSuccess) return set_error(MP_ECUDA, "stream sync: %s", cudaGetErrorString(e));
    return MP_OK;
}

// ------------------------------------------------------------ autotuner
namespace {

__global__ void fill_test_kernel(void *A, int64_t n, int dtype, uint32_t seed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u ^ seed;
        h ^= h >> 13;
        h *= 0x5bd1e995u;
        h ^= h >> 15;
        const uint32_t v = (h & 7) == 0 ? (dtype == MP_I16 ? 0x7FFFu : 0xFFu) : (h >> 8) & 31;
        if (dtype == MP_I16) ((uint16_t *)A)[i] = (uint16_t)v;
        else ((uint8_t *)A)[i] = (uint8_t)v;
    }
}

}  // namespace

int autotune(int32_t *table_out) {
    static const int64_t sizes[kClasses] = {96, 192, 384, 768, 1536, 3072};
    TuneTable t = default_table();
    const int64_t nmax = sizes[kClasses - 1];
    DevBuf buf;
    MP_TRY(buf.alloc((size_t)nmax * nmax * 2 * 3, nullptr, true));
    cudaEvent_t e0, e1;
    MP_CUDA_TRY(cudaEventCreate(&e0));
    MP_CUDA_TRY(cudaEventCreate(&e1));
    for (int d = 0; d < 2; ++d) {
        const int dtype = d == 0 ? MP_I16 : MP_U8;
        const size_t es = d == 0 ? 2 : 1;
        for (int c = 0; c < kClasses; ++c) {
            const int64_t n = sizes[c];
            uint8_t *X = buf.as<uint8_t>(), *Y = X + (size_t)n * n * es, *Z = Y + (size_t)n * n * es;
            fill_test_kernel<<<256, 256>>>(X, n * n, dtype, 17u + c);
            fill_test_kernel<<<256, 256>>>(Y, n * n, dtype, 91u + c);
            float best = 1e30f;
            for (int cfg = 0; cfg < 2; ++cfg) {
                float bt = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    MP_CUDA_TRY(cudaEventRecord(e0));
                    int rc = dtype == MP_I16
                                 ? run_dense<uint16_t>((uint16_t *)X, (uint16_t *)Y, (uint16_t *)Z, n, n, n,
                                                       n, n, n, nullptr, cfg, nullptr)
                                 : run_dense<uint8_t>(X, Y, Z, n, n, n, n, n, n, nullptr, cfg, nullptr);
                    if (rc != MP_OK) return rc;
                    MP_CUDA_TRY(cudaEventRecord(e1));
                    MP_CUDA_TRY(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    MP_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                    bt = std::min(bt, ms);
                }
                if (bt < best) {
                    best = bt;
                    t.cfg[d][c] = cfg;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int dev = -1;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[dev] = t;
    }
    if (table_out) memcpy(table_out, &t.cfg[0][0], sizeof t.cfg);
    return MP_OK;
}

int tuning_set(const int32_t *table) {
    TuneTable t;
    for (int d = 0; d < 2; ++d)
        for (int c = 0; c < kClasses; ++c) {
            const int32_t v = table[d * kClasses + c];
            if (v != 0 && v != 1) return set_error(MP_EINVAL, "tile shape %d not 0 or 1", v);
            t.cfg[d][c] = v;
        }
    int dev = -1;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[dev] = t;
    return MP_OK;
}

int tuning_get(int32_t *table) {
    TuneTable t;
    MP_TRY(current_table(&t));
    memcpy(table, &t.cfg[0][0], sizeof t.cfg);
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

// Device address of g_noalloc_masks on the current device, looked up with
// that device current the first time a device is used.  In host code the
// array's name is only a host-side stand-in, never a device address.  A
// cudaDeviceReset unloads the module, so a cached address is checked on
// every call and looked up again once it no longer names device memory of
// this device.
int noalloc_scratch(uint8_t **out) {
    int dev = -1;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return set_error(MP_EINVAL, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_addr[dev]) {
        cudaPointerAttributes at;
        const cudaError_t e = cudaPointerGetAttributes(&at, g_noalloc_addr[dev]);
        if (e != cudaSuccess || at.type != cudaMemoryTypeDevice || at.device != dev) {
            cudaGetLastError();
            g_noalloc_addr[dev] = nullptr;
        }
    }
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

// Operands are read in place: rows off the 8-element grid take the product
// kernel's scalar-load path instead of being repacked (a repack would need
// memory).
template <typename T>
int run_dense_noalloc(const T *X, const T *Y, T *Z, int64_t M, int64_t N, int64_t K,
                      int64_t ldx, int64_t ldy, int64_t ldz, cudaStream_t s) {
    const int64_t mb = (M + MASK_BLOCK - 1) / MASK_BLOCK, nb = (N + MASK_BLOCK - 1) / MASK_BLOCK;
    const int64_t kb = (K + MASK_BLOCK - 1) / MASK_BLOCK;
    const uint8_t *xm = nullptr, *ym = nullptr;
    if (K > 0) {
        uint8_t *base = nullptr;
        MP_TRY(noalloc_scratch(&base));
        // every mask byte the product reads is written here first, so stale
        // contents of an earlier call never matter
        uint8_t *xmw = base, *ymw = base + mb * kb;
        block_mask_kernel<T><<<dim3((unsigned)kb, (unsigned)mb), 256, 0, s>>>(X, M, K, ldx, xmw, kb,
                                                                           nullptr, 0);
        block_mask_kernel<T><<<dim3((unsigned)nb, (unsigned)kb), 256, 0, s>>>(Y, K, N, ldy, ymw, nb,
                                                                           nullptr, 0);
        MP_CUDA_TRY(cudaGetLastError());
        xm = xmw;
        ym = ymw;
    }
    return launch_product<T>(make_args<T>(X, Y, Z, M, N, K, ldx, ldy, ldz, xm, ym, nullptr), 0, s);
}

}  // namespace

int dense_minplus_noalloc(const void *X, const void *Y, void *Z, int64_t M, int64_t N,
                          int64_t K, int64_t ldx, int64_t ldy, int64_t ldz, int dtype,
                          cudaStream_t s) {
    if (M == 0 || N == 0) return MP_OK;
    const int64_t mb = (M + MASK_BLOCK - 1) / MASK_BLOCK, nb = (N + MASK_BLOCK - 1) / MASK_BLOCK;
    const int64_t kb = (K + MASK_BLOCK - 1) / MASK_BLOCK;
    if (mb > 65535)
        return set_error(MP_EINVAL, "M = %lld too large for one launch", (long long)M);
    // in double: the block counts are below 2^57, their products may not fit int64
    const double need = (double)mb * (double)kb + (double)kb * (double)nb;
    if (need > (double)kNoAllocMaskBytes)
        return set_error(MP_EINVAL,
                         "problem needs %.0f mask bytes; the fixed scratch holds %zu "
                         "(ceil(M/128)*ceil(K/128) + ceil(K/128)*ceil(N/128) must not exceed it)",
                         need, kNoAllocMaskBytes);
    if (dtype == MP_I16)
        return run_dense_noalloc<uint16_t>((const uint16_t *)X, (const uint16_t *)Y,
                                           (uint16_t *)Z, M, N, K, ldx, ldy, ldz, s);
    if (dtype == MP_U8)
        return run_dense_noalloc<uint8_t>((const uint8_t *)X, (const uint8_t *)Y, (uint8_t *)Z,
                                          M, N, K, ldx, ldy, ldz, s);
    return set_error(MP_EINVAL, "unknown dtype %d", dtype);
}

}  // namespace mp
