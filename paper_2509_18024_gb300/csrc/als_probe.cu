// Roofline probes: the peak rates this library's kernels are measured
// against, timed on the device with CUDA events around one launch (after a
// warm-up launch). Each probe allocates its own buffers, so nothing of a
// handle is involved.
//   FFMA / DFMA   FP32 / FP64 fused multiply-add throughput of the SMs
//                 (independent chains per thread; 2 flops per FMA)
//   TC_BF16 / TC_TF32  tcgen05.mma throughput, one CTA per SM issuing
//                 M = 128, N = 256 MMAs back to back from shared memory into a
//                 tensor-memory accumulator (2 M N K flops each)
//   L2_GATHER     bytes/s of random 128-byte row gathers from a 16 MB factor
//                 that stays in L2 (the gather of a design slice)
//   HBM_COPY      bytes/s (read + write) of a 4 GB device-to-device copy kernel
#include <cuda_runtime.h>
#include <stdint.h>

#include "core_als.h"
#include "als_tc.cuh"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_probe_ffma(int64_t iters, float seed, float* sink) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
    const float m = 0.999999f, d = 1e-7f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, d);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678f) sink[blockIdx.x] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(256) k_probe_dfma(int64_t iters, double seed, double* sink) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (double)(threadIdx.x + c);
    const double m = 0.999999, d = 1e-7;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, d);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678) sink[blockIdx.x] = s;
}

// tcgen05 throughput: one thread issues `batches` x 8 MMAs (N = 256) into one
// accumulator, committing each batch to an mbarrier; the CTA waits (bounded)
// for the last commit. Operands are zero tiles in the K-major no-swizzle
// layout of als_tc.cuh.
constexpr int kTcN = 256, kTcM = 128;
template <int PREC>
__global__ void __launch_bounds__(128, 1) k_probe_tc(int64_t batches, unsigned* err) {
    using namespace als;
    constexpr int ESZ = PREC == TC_BF16 ? 2 : 4;
    constexpr int KSTEP = 32 / ESZ;                      // K of one MMA (32 bytes)
    constexpr int A_BYTES = kTcM * 32, B_BYTES = kTcN * 32;
    constexpr uint32_t IDESC = (1u << 4) | ((PREC == TC_BF16 ? 1u : 2u) << 7) | ((PREC == TC_BF16 ? 1u : 2u) << 10) |
                               ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
    __shared__ __align__(1024) uint8_t tiles[A_BYTES + B_BYTES];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int e = tid; e < (A_BYTES + B_BYTES) / 16; e += blockDim.x)
        reinterpret_cast<uint4*>(tiles)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"((uint32_t)kTcN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    if (tid == 0) {
        const uint64_t ad = umma_desc(smem_addr(tiles), (kTcM / 8) * 128, 128);
        const uint64_t bd = umma_desc(smem_addr(tiles + A_BYTES), (kTcN / 8) * 128, 128);
        uint32_t phase = 0;
        bool ok = true;
        // Batch b's MMAs are queued before the wait for batch b - 1's commit,
        // and b is committed after it, so at most one commit is outstanding
        // at any wait (no phase can be skipped).
        for (int64_t b = 0; b < batches && ok; ++b) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint32_t accum = (b > 0 || q > 0) ? 1u : 0u;
                if (PREC == TC_BF16)
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(IDESC), "r"(accum));
                else
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(IDESC), "r"(accum));
            }
            if (b > 0) {
                ok = mbar_wait(&bar, phase);
                phase ^= 1u;
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&bar)));
        }
        if (ok) ok = mbar_wait(&bar, phase);
        if (!ok) report_timeout(err);
        s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    (void)KSTEP;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTcN));
}

// Random 128-byte row gathers (8 threads per row, one float4 each).
__global__ void __launch_bounds__(256) k_probe_gather(const float4* __restrict__ Y, const int32_t* __restrict__ idx,
                                                      int64_t n_idx, float* sink) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t total = n_idx * 8;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = __ldg(Y + (int64_t)idx[g >> 3] * 8 + (g & 7));
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
    }
    if (acc.x + acc.y + acc.z + acc.w == 12345.678f) sink[0] = acc.x;
}

__global__ void __launch_bounds__(256) k_probe_copy(const float4* __restrict__ src, float4* __restrict__ dst, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = src[e];
}

__global__ void k_probe_fill_idx(int32_t* idx, int64_t n, int64_t rows) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = (uint64_t)e * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        idx[e] = (int32_t)(z % (uint64_t)rows);
    }
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

}  // namespace

extern "C" int als_probe(int kind, double* value_host, double* ms_host, void* cuda_stream) {
    if (!value_host) return ALS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess) {
        cudaGetLastError();
        return ALS_ERR_CUDA;
    }
    Timer t;
    void* buf = nullptr;
    void* buf2 = nullptr;
    double work = 0.0;  // flops or bytes of the timed launch
    int rc = ALS_OK;
    float ms = 0.f;
    auto timed = [&](auto launch) {
        launch();  // warm-up
        cudaEventRecord(t.a, st);
        launch();
        cudaEventRecord(t.b, st);
        if (cudaEventSynchronize(t.b) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = ALS_ERR_CUDA;
        cudaEventElapsedTime(&ms, t.a, t.b);
    };
    switch (kind) {
        case ALS_PROBE_FFMA: {
            if (cudaMalloc(&buf, 4096 * 4) != cudaSuccess) return ALS_ERR_OOM;
            const int grid = n_sm * 8;
            const int64_t iters = 1 << 16;
            work = 2.0 * kChains * iters * 256.0 * grid;
            timed([&] { k_probe_ffma<<<grid, 256, 0, st>>>(iters, 1.0f, static_cast<float*>(buf)); });
            break;
        }
        case ALS_PROBE_DFMA: {
            if (cudaMalloc(&buf, 4096 * 8) != cudaSuccess) return ALS_ERR_OOM;
            const int grid = n_sm * 8;
            const int64_t iters = 1 << 11;
            work = 2.0 * kChains * iters * 256.0 * grid;
            timed([&] { k_probe_dfma<<<grid, 256, 0, st>>>(iters, 1.0, static_cast<double*>(buf)); });
            break;
        }
        case ALS_PROBE_TC_BF16:
        case ALS_PROBE_TC_TF32: {
            if (cudaMalloc(&buf, 16) != cudaSuccess) return ALS_ERR_OOM;
            cudaMemsetAsync(buf, 0, 16, st);
            const bool bf = kind == ALS_PROBE_TC_BF16;
            const int64_t batches = bf ? 20000 : 10000;
            const double k_per = bf ? 16.0 : 8.0;
            work = 2.0 * kTcM * kTcN * k_per * 8.0 * batches * n_sm;
            unsigned* err = static_cast<unsigned*>(buf);
            if (bf)
                timed([&] { k_probe_tc<als::TC_BF16><<<n_sm, 128, 0, st>>>(batches, err); });
            else
                timed([&] { k_probe_tc<als::TC_TF32><<<n_sm, 128, 0, st>>>(batches, err); });
            unsigned e = 0;
            if (rc == ALS_OK && cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost) == cudaSuccess && e) rc = ALS_ERR_TIMEOUT;
            break;
        }
        case ALS_PROBE_L2_GATHER: {
            const int64_t rows = 131072;            // 16 MB of 128-byte rows
            const int64_t n_idx = 1 << 24;          // 2 GB gathered
            if (cudaMalloc(&buf, rows * 128) != cudaSuccess) return ALS_ERR_OOM;
            if (cudaMalloc(&buf2, n_idx * 4 + 64) != cudaSuccess) {
                cudaFree(buf);
                return ALS_ERR_OOM;
            }
            cudaMemsetAsync(buf, 0, rows * 128, st);
            int32_t* idx = static_cast<int32_t*>(buf2);
            k_probe_fill_idx<<<4096, 256, 0, st>>>(idx, n_idx, rows);
            work = (double)n_idx * 128.0;
            float* sink = reinterpret_cast<float*>(static_cast<char*>(buf2) + n_idx * 4);
            timed([&] {
                k_probe_gather<<<n_sm * 8, 256, 0, st>>>(static_cast<const float4*>(buf), idx, n_idx, sink);
            });
            break;
        }
        case ALS_PROBE_HBM_COPY: {
            const int64_t bytes = (int64_t)2 << 30;  // 2 GB read + 2 GB written
            if (cudaMalloc(&buf, bytes) != cudaSuccess) return ALS_ERR_OOM;
            if (cudaMalloc(&buf2, bytes) != cudaSuccess) {
                cudaFree(buf);
                return ALS_ERR_OOM;
            }
            cudaMemsetAsync(buf, 0, bytes, st);
            work = 2.0 * (double)bytes;
            timed([&] {
                k_probe_copy<<<n_sm * 16, 256, 0, st>>>(static_cast<const float4*>(buf), static_cast<float4*>(buf2),
                                                        bytes / 16);
            });
            break;
        }
        default:
            return ALS_ERR_ARG;
    }
    cudaStreamSynchronize(st);
    if (buf) cudaFree(buf);
    if (buf2) cudaFree(buf2);
    if (rc) return rc;
    // TFLOP/s for the arithmetic probes, GB/s for the memory probes.
    const double s = (double)ms / 1e3;
    const bool bytes_probe = kind == ALS_PROBE_L2_GATHER || kind == ALS_PROBE_HBM_COPY;
    *value_host = s > 0 ? work / s / (bytes_probe ? 1e9 : 1e12) : 0.0;
    if (ms_host) *ms_host = ms;
    return ALS_OK;
}
