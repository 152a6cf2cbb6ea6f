// K3: reductions that read gamma_2 off the powers.
//
// Theorem 2: gamma_2(P_n x C_m) = min_i (A^m)_ii.  diag_min reads the
// diagonal of one stored power.  min_trace gives min_i (X (x) Y)_ii =
// min_{i,l} X_il + Y_li without forming the product: it is what the
// repeated-squaring path uses for the last two factors of A^m.  Both reduce
// in registers, then across the warp with shuffles, then one atomicMin per
// warp into a 32-bit result that starts at INF.
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

}  // namespace

int launch_fill_i32(int32_t *p, int64_t count, int32_t v, cudaStream_t s) {
    if (count <= 0) return MP_OK;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    fill_i32_kernel<<<(unsigned)blocks, 256, 0, s>>>(p, count, v);
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
