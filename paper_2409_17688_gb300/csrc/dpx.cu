// K6: throughput microbenchmark of the packed 16-bit min / add-min
// instructions the (min,+) kernels are built on.  Every thread of a full
// grid (8 CTAs of 256 threads per SM) runs 8 independent dependency chains,
// so issue, not latency, limits the rate.  The measured rate is the
// denominator of the "fraction of DPX peak" that the benchmark reports.
//
// variant 0: __viaddmin_u16x2 -- one (min,+) term per 16-bit lane, 2 per instruction
// variant 1: __vimin3_u16x2   -- two gathered values per lane, 4 terms per instruction
// variant 2: __vminu2         -- one value per lane, 2 terms per instruction
// variant 3: shared-memory loads -- 16-byte ld.shared per lane, conflict-free
//            (a warp's 512 bytes cover all 32 banks four times); the rate is
//            in bytes per second, the roof of the shared-memory-bound kernels
#include "mp_internal.cuh"

namespace mp {

namespace {

template <int V>
__global__ void __launch_bounds__(256) dpx_peak_kernel(int64_t iters, uint32_t seed,
                                                       uint32_t *sink) {
    uint32_t a[8], b[8];
    const uint32_t y = (seed ^ threadIdx.x) & 0x00FF00FFu;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        a[j] = (seed * (j + 3) + threadIdx.x) & 0x3FFF3FFFu;
        b[j] = (seed * (j + 7) + blockIdx.x) & 0x3FFF3FFFu;
    }
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (V == 0) {
                a[j] = __viaddmin_u16x2(b[j], y, a[j]);
                b[j] = __viaddmin_u16x2(a[j], y, b[j]);
            } else if (V == 1) {
                a[j] = __vimin3_u16x2(a[j], b[j], y);
                b[j] = __vimin3_u16x2(b[j], a[j], y ^ 0x00010001u);
            } else {
                a[j] = __vminu2(a[j], b[j] ^ y);
                b[j] = __vminu2(b[j], a[j] ^ y);
            }
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) r ^= a[j] ^ b[j];
    if (r == seed) sink[0] = r;  // keeps the chains alive; practically never taken
}

constexpr int kSmemProbeBytes = 16384;  // per CTA; 8 CTAs per SM use 128 KB

// Eight independent 16-byte loads per iteration per thread; consecutive
// lanes read consecutive 16-byte words, so every quarter warp touches the 32
// banks once (no conflicts) and a warp's load is four wavefronts.  The XOR
// of everything read keeps the loads alive.
__global__ void __launch_bounds__(256) smem_peak_kernel(int64_t iters, uint32_t seed, uint32_t *sink) {
    __shared__ __align__(16) uint32_t buf[kSmemProbeBytes / 4];
    for (int i = threadIdx.x; i < kSmemProbeBytes / 4; i += blockDim.x) buf[i] = seed * (uint32_t)i;
    __syncthreads();
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
    uint32_t acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
    // 16 bytes per lane, the warp's 512 bytes start on a 512-byte boundary
    uint32_t off = (uint32_t)threadIdx.x * 16u;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t x, y, z, w;
            // eight distinct 512-byte segments, 2 KB apart
            const uint32_t a = base + ((off + (uint32_t)j * 2048u) & (kSmemProbeBytes - 1));
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(x), "=r"(y), "=r"(z), "=r"(w)
                         : "r"(a));
            acc0 ^= x;
            acc1 ^= y;
            acc2 ^= z;
            acc3 ^= w;
        }
        off += 512u;
    }
    if ((acc0 ^ acc1 ^ acc2 ^ acc3) == seed) sink[0] = acc0;  // practically never taken
}

}  // namespace

int dpx_peak(int variant, int64_t iters, double *ops_per_s) {
    if (variant < 0 || variant > 3 || iters < 1)
        return set_error(MP_EINVAL, "dpx_peak: variant 0..3 and iters >= 1");
    DeviceInfo di;
    MP_TRY(device_info(&di));
    DevBuf sink;
    MP_TRY(sink.alloc(16, nullptr, true));
    const int blocks = di.sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    MP_CUDA_TRY(cudaEventCreate(&e0));
    MP_CUDA_TRY(cudaEventCreate(&e1));
    auto launch = [&](int64_t it) {
        if (variant == 3) smem_peak_kernel<<<blocks, threads>>>(it, 12345u, sink.as<uint32_t>());
        else if (variant == 0) dpx_peak_kernel<0><<<blocks, threads>>>(it, 12345u, sink.as<uint32_t>());
        else if (variant == 1) dpx_peak_kernel<1><<<blocks, threads>>>(it, 12345u, sink.as<uint32_t>());
        else dpx_peak_kernel<2><<<blocks, threads>>>(it, 12345u, sink.as<uint32_t>());
    };
    launch(64);  // warm-up
    MP_CUDA_TRY(cudaEventRecord(e0));
    launch(iters);
    MP_CUDA_TRY(cudaEventRecord(e1));
    MP_CUDA_TRY(cudaEventSynchronize(e1));
    MP_CUDA_TRY(cudaGetLastError());
    float ms = 0.f;
    MP_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (variant == 3) {
        // 8 loads of 16 bytes per thread and iteration
        *ops_per_s = (double)blocks * threads * (double)iters * 8.0 * 16.0 / (ms * 1e-3);
        return MP_OK;
    }
    const double instr = (double)blocks * threads * (double)iters * 16.0;  // 8 chains x 2 per iteration
    const double per_instr = variant == 1 ? 4.0 : 2.0;
    *ops_per_s = instr * per_instr / (ms * 1e-3);
    return MP_OK;
}

}  // namespace mp
