// K3: reductions that read gamma_2 off the powers.
//
// Theorem 2: gamma_2(P_n x C_m) = min_i (A^m)_ii.  diag_min reads the
// diagonal of one stored power.  min_trace gives min_i (X (x) Y)_ii =
// min_{i,l} X_il + Y_li without forming the product: it is what the
// repeated-squaring path uses for the last two factors of A^m.  Both reduce
// in registers, then across the warp with shuffles, then one atomicMin per
// warp into a 32-bit result that starts at INF.
#include <algorithm>
#include <cstring>

#include "mp_internal.cuh"

namespace mp {

namespace {

__device__ __forceinline__ int32_t warp_min(int32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

__global__ void fill_i32_kernel(int32_t *p, int64_t count, int32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// g[0 .. k_max) of up to kGdiagChains chains: g[0] from the chain's first
// power (a value kept on the device), INF for the powers still to come.
struct GdiagInitArgs {
    int32_t *dst[kGdiagChains];
    const int32_t *g1[kGdiagChains];
    int count, k_max;
};
__global__ void gdiag_init_kernel(const __grid_constant__ GdiagInitArgs a) {
    for (int c = 0; c < a.count; ++c)
        for (int i = (int)threadIdx.x; i < a.k_max; i += (int)blockDim.x)
            a.dst[c][i] = i == 0 ? *a.g1[c] : (int32_t)kInf16;
}

__global__ void diag_min_kernel(const int16_t *__restrict__ P, int64_t N, int64_t ld,
                                int32_t *out) {
    int32_t v = (int32_t)kInf16;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        v = min(v, (int32_t)(uint16_t)P[i * ld + i]);
    v = warp_min(v);
    if ((threadIdx.x & 31) == 0 && v < (int32_t)kInf16) atomicMin(out, v);
}

// One 32 x 32 tile (i-block I, l-block L) per CTA: X[I][L] is read by rows,
// Y[L][I] by rows into shared memory, and the pairs X_il + Y_li are formed
// through the transposed shared tile.
__global__ void min_trace_kernel(const int16_t *__restrict__ X, const int16_t *__restrict__ Y,
                                 int64_t N, int64_t ldx, int64_t ldy, int32_t *out) {
    __shared__ int32_t ys[32][33];
    const int64_t i0 = (int64_t)blockIdx.y * 32, l0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int r = ty; r < 32; r += 8) {
        int64_t l = l0 + r, i = i0 + tx;
        ys[r][tx] = (l < N && i < N) ? (int32_t)(uint16_t)Y[l * ldy + i] : (int32_t)kInf16;
    }
    __syncthreads();
    int32_t v = 2 * (int32_t)kInf16;
    for (int r = ty; r < 32; r += 8) {
        int64_t i = i0 + r, l = l0 + tx;
        int32_t x = (i < N && l < N) ? (int32_t)(uint16_t)X[i * ldx + l] : (int32_t)kInf16;
        v = min(v, x + ys[tx][r]);
    }
    v = min(warp_min(v), (int32_t)kInf16);
    if (tx == 0 && v < (int32_t)kInf16) atomicMin(out, v);
}

__global__ void set_one_kernel(int32_t *out, int32_t v) { *out = v; }

// K4: is X - Y a constant matrix (Algorithms 3 and 4)?  out[0] = min and
// out[1] = max of X - Y over entries finite in both, out[2] = 1 when some
// entry is INF in exactly one of them, out[3] = 1 when some entry is finite
// in both.  The difference is constant exactly when out[2] = 0, out[3] = 1
// and out[0] = out[1].
__global__ void diff_init_kernel(int32_t *out) {
    out[0] = 0x7FFFFFFF;
    out[1] = (int32_t)0x80000000;
    out[2] = 0;
    out[3] = 0;
}

__global__ void diff_init_many_kernel(int32_t *out, int64_t count4) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count4) return;
    out[4 * i] = 0x7FFFFFFF;
    out[4 * i + 1] = (int32_t)0x80000000;
    out[4 * i + 2] = 0;
    out[4 * i + 3] = 0;
}

__global__ void diff_const_kernel(const int16_t *__restrict__ X, const int16_t *__restrict__ Y,
                                  int64_t count, int32_t *out) {
    int32_t lo = 0x7FFFFFFF, hi = (int32_t)0x80000000, mism = 0, fin = 0;
    const int64_t n2 = count / 2;
    const uint32_t *x2 = reinterpret_cast<const uint32_t *>(X);
    const uint32_t *y2 = reinterpret_cast<const uint32_t *>(Y);
    const bool vec = ((uintptr_t)X % 4 == 0) && ((uintptr_t)Y % 4 == 0);
    auto one = [&](uint32_t a, uint32_t b) {
        const bool fa = a < kInf16, fb = b < kInf16;
        if (fa != fb) mism = 1;
        if (fa && fb) {
            const int32_t d = (int32_t)a - (int32_t)b;
            lo = min(lo, d);
            hi = max(hi, d);
            fin = 1;
        }
    };
    if (vec) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
             i += (int64_t)gridDim.x * blockDim.x) {
            const uint32_t a = x2[i], b = y2[i];
            one(a & 0xFFFFu, b & 0xFFFFu);
            one(a >> 16, b >> 16);
        }
        if (count & 1) {
            if (blockIdx.x == 0 && threadIdx.x == 0)
                one((uint16_t)X[count - 1], (uint16_t)Y[count - 1]);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
             i += (int64_t)gridDim.x * blockDim.x)
            one((uint16_t)X[i], (uint16_t)Y[i]);
    }
    lo = warp_min(lo);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
        mism |= __shfl_xor_sync(0xFFFFFFFFu, mism, o);
        fin |= __shfl_xor_sync(0xFFFFFFFFu, fin, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (fin) {
            atomicMin(&out[0], lo);
            atomicMax(&out[1], hi);
            atomicOr(&out[3], 1);
        }
        if (mism) atomicOr(&out[2], 1);
    }
}

}  // namespace

int launch_fill_i32(int32_t *p, int64_t count, int32_t v, cudaStream_t s) {
    if (count <= 0) return MP_OK;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    fill_i32_kernel<<<(unsigned)blocks, 256, 0, s>>>(p, count, v);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int launch_gdiag_init(int32_t *const *dst, const int32_t *const *g1, int count, int k_max,
                      cudaStream_t s) {
    if (count < 0 || count > kGdiagChains) return set_error(MP_EINVAL, "%d chains for one g init", count);
    if (count == 0 || k_max < 1) return MP_OK;
    GdiagInitArgs a;
    memset(&a, 0, sizeof(a));
    for (int c = 0; c < count; ++c) {
        a.dst[c] = dst[c];
        a.g1[c] = g1[c];
    }
    a.count = count;
    a.k_max = k_max;
    gdiag_init_kernel<<<1, 256, 0, s>>>(a);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int launch_diag_min(const int16_t *P, int64_t N, int64_t ld, int32_t *out, bool init,
                    cudaStream_t s) {
    if (init) {
        set_one_kernel<<<1, 1, 0, s>>>(out, (int32_t)kInf16);
        MP_CUDA_TRY(cudaGetLastError());
    }
    if (N <= 0) return MP_OK;
    int64_t blocks = (N + 255) / 256;
    if (blocks > 256) blocks = 256;
    diag_min_kernel<<<(unsigned)blocks, 256, 0, s>>>(P, N, ld, out);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int launch_diff_const(const int16_t *X, const int16_t *Y, int64_t count, int32_t *out,
                      cudaStream_t s, bool init) {
    if (init) {
        diff_init_kernel<<<1, 1, 0, s>>>(out);
        MP_CUDA_TRY(cudaGetLastError());
    }
    if (count <= 0) return MP_OK;
    DeviceInfo di;
    MP_TRY(device_info(&di));
    int64_t blocks = (count / 2 + 255) / 256;
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)di.sms * 8));
    diff_const_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, Y, count, out);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int launch_diff_init(int32_t *out, int64_t count4, cudaStream_t s) {
    if (count4 <= 0) return MP_OK;
    diff_init_many_kernel<<<(unsigned)((count4 + 255) / 256), 256, 0, s>>>(out, count4);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int launch_min_trace(const int16_t *X, const int16_t *Y, int64_t N, int64_t ldx, int64_t ldy,
                     int32_t *out, cudaStream_t s) {
    set_one_kernel<<<1, 1, 0, s>>>(out, (int32_t)kInf16);
    MP_CUDA_TRY(cudaGetLastError());
    if (N <= 0) return MP_OK;
    int64_t nb = (N + 31) / 32;
    if (nb > 65535) return set_error(MP_EINVAL, "N = %lld too large for min_trace", (long long)N);
    min_trace_kernel<<<dim3((unsigned)nb, (unsigned)nb), 256, 0, s>>>(X, Y, N, ldx, ldy, out);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace mp
