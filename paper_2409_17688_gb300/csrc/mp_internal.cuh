// Internal helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>

#include <stdarg.h>

#include <string>
#include <vector>

#include "../../include/minplus.h"

namespace mp {

// ---------------------------------------------------------------- errors
int set_error(int code, const char *fmt, ...);
const char *last_error();

#define MP_CUDA_TRY(expr)                                                          \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess)                                                     \
            return ::mp::set_error(MP_ECUDA, "%s failed: %s (%s:%d)", #expr,       \
                                   cudaGetErrorString(_e), __FILE__, __LINE__);    \
    } while (0)

#define MP_TRY(expr)                   \
    do {                               \
        int _s = (expr);               \
        if (_s != MP_OK) return _s;    \
    } while (0)

// NVTX range over a scope of host code (a no-op unless a profiler is
// attached), named with printf-style arguments.
struct NvtxScope {
    explicit NvtxScope(const char *fmt, ...) {
        char buf[96];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        nvtxRangePushA(buf);
    }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

// ------------------------------------------------------------ constants
constexpr uint32_t kInf16 = 0x7FFFu;
constexpr uint32_t kInf16x2 = 0x7FFF7FFFu;
constexpr uint32_t kInf8 = 0xFFu;

// Bounds-checked builds (-DMP_CHECK): mp_ix(i, n, status) is i where i < n;
// otherwise it latches MP_ECHECK in the device status word (the first error
// wins) and gives 0, so that the access it feeds stays inside its buffer and
// the kernel runs to its end.  Without MP_CHECK it is i itself.
template <class T>
__device__ __forceinline__ T mp_ix(T i, T n, int *status) {
#ifdef MP_CHECK
    if (!(i < n)) {
        if (status) atomicCAS(status, 0, MP_ECHECK);
        return T(0);
    }
#else
    (void)n;
    (void)status;
#endif
    return i;
}

// Bound on spin iterations of any device-side wait (mbarrier phases).  A
// wait that runs out latches MP_ETIMEOUT into the device status word and
// the kernel returns without touching the stalled buffer.
constexpr uint32_t kSpinLimit = 1u << 26;

// Per-device status word, set by kernels on a bounded-wait timeout.
int device_status_ptr(int **p);

// ------------------------------------------------------ device properties
struct DeviceInfo {
    int device = -1;
    int sms = 0;
    size_t smem_optin = 0;  // dynamic shared memory one block may take
    size_t smem_sm = 0;     // shared memory of one SM
};
int device_info(DeviceInfo *out);

// ------------------------------------------------------- stream-ordered memory
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    bool persistent = false;  // plain cudaMalloc, for buffers that outlive a call
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) {
            if (persistent) cudaFree(p);
            else cudaFreeAsync(p, s);
        }
        p = nullptr;
        bytes = 0;
    }
    int alloc(size_t n, cudaStream_t st, bool keep = false) {
        release();
        s = st;
        bytes = n;
        persistent = keep;
        if (n == 0) return MP_OK;
        cudaError_t e = keep ? cudaMalloc(&p, n) : cudaMallocAsync(&p, n, st);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return set_error(MP_ENOMEM, "device allocation of %zu bytes failed: %s", n,
                             cudaGetErrorString(e));
        }
        return MP_OK;
    }
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

inline bool ranges_overlap(const void *a, size_t an, const void *b, size_t bn) {
    if (!a || !b || an == 0 || bn == 0) return false;
    uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + bn && b0 < a0 + an;
}

// Bytes spanned by a rows x cols matrix with leading dimension ld.
inline size_t span_bytes(int64_t rows, int64_t cols, int64_t ld, size_t elem) {
    if (rows <= 0 || cols <= 0) return 0;
    return ((size_t)(rows - 1) * (size_t)ld + (size_t)cols) * elem;
}

// ----------------------------------------------------------- words (a1)
// Correct n-words in lexicographic order, packed 2 bits per letter with
// letter 1 in the top pair.  Host only.
void enumerate_words(int n, std::vector<uint32_t> *out);

// Per-word letter masks for the device arc test: bit i <-> letter i+1.
struct WordMasks {
    uint16_t zero, one, two, pad;
};
void word_masks(int n, const std::vector<uint32_t> &words, std::vector<WordMasks> *out);
// partner[c] = index of word c read backwards (an involution of the words).
int mirror_words(int n, const std::vector<uint32_t> &words, std::vector<int64_t> *partner);

// ------------------------------------------------------- kernels (launchers)
int launch_build_transfer(int n, const WordMasks *d_masks, int64_t N, int16_t *A,
                          int64_t lda, cudaStream_t s);
int launch_transfer_csr_count(int n, const WordMasks *d_masks, int64_t N, int64_t *counts,
                              cudaStream_t s);
int launch_transfer_csr_fill(int n, const WordMasks *d_masks, int64_t N, const int64_t *row_ptr,
                             int32_t *col, cudaStream_t s);
int launch_fill_i32(int32_t *p, int64_t count, int32_t v, cudaStream_t s);
// dst[c][0] = *g1[c] and dst[c][1 .. k_max) = INF for count <= kGdiagChains chains, one launch.
constexpr int kGdiagChains = 8;
int launch_gdiag_init(int32_t *const *dst, const int32_t *const *g1, int count, int k_max,
                      cudaStream_t s);
int launch_diag_min(const int16_t *P, int64_t N, int64_t ld, int32_t *out, bool init,
                    cudaStream_t s);
// init false: fold into out[0..4) as it stands (statistics over several
// blocks of columns); launch_diff_init resets count4 groups of four.
int launch_diff_const(const int16_t *X, const int16_t *Y, int64_t count, int32_t *out,
                      cudaStream_t s, bool init = true);
int launch_diff_init(int32_t *out, int64_t count4, cudaStream_t s);
int launch_min_trace(const int16_t *X, const int16_t *Y, int64_t N, int64_t ldx,
                     int64_t ldy, int32_t *out, cudaStream_t s);
// The transfer chain of A(D_n) with a caller-chosen slot stride (elements).
int transfer_powers_strided(int n, int k_max, int16_t *powers_opt, size_t slot,
                            int32_t *gdiag_opt, cudaStream_t s);
// Dense (min,+) product; gdiag (optional) gets atomicMin of the diagonal.
int dense_minplus(const void *X, const void *Y, void *Z, int64_t M, int64_t N,
                  int64_t K, int64_t ldx, int64_t ldy, int64_t ldz, int dtype,
                  int32_t *gdiag, cudaStream_t s);

}  // namespace mp
