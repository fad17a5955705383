// Pipe-throughput probes (not an operation of the paper): the denominators of
// the library's roofline fractions measured on the running GPU rather than
// derived from unit counts.
//
//   kind 0: FP64 FMA    -- independent fma chains per thread, all SMs
//   kind 1: FP32 FMA    -- the same in float (the pipe of the mixed path's
//                          float-float kernels)
//   kind 2: TF32 tensor -- tcgen05.mma kind::tf32, M = 128, N = 256, K = 8,
//                          issued back to back by one thread per CTA (one CTA
//                          per SM) into one tensor-memory accumulator, operands
//                          in shared memory (the LU update's instruction and
//                          descriptor forms, tc_update.cuh); completion by
//                          tcgen05.commit on an mbarrier with a bounded wait
// Each is timed with CUDA events around one launch after a warm-up launch.
#include <cstdint>

#include "internal.h"
#include "tcgen05_util.cuh"

namespace pmlbie {
namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T seed, T* sink) {
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
    const T m = (T)0.999999, k = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == (T)12345.678) sink[threadIdx.x] = s;   // keeps the chains alive
}

constexpr int kProbeN = 256;                          // MMA N (columns, TMEM columns)
constexpr uint32_t kProbeIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kProbeN >> 3) << 17) |
                                 ((uint32_t)(128 >> 4) << 24);
constexpr uint32_t kProbeA = 128 * 8 * 4;             // A: 128 x 8 tf32, K-major
constexpr uint32_t kProbeB = kProbeN * 8 * 4;         // B: 256 x 8 tf32, K-major
constexpr uint32_t kProbeSmem = kProbeA + kProbeB + 4096 + 64;
// launch size: enough shared memory that one CTA occupies an SM
constexpr uint32_t kProbeSmemLaunch = 120 * 1024;

__global__ void __launch_bounds__(128, 1) tf32_probe_kernel(int iters, int* status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* sA = sm;
    unsigned char* sB = sA + kProbeA;
    unsigned char* tail = sB + kProbeB + 4096;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(tail);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tail + 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    // operands: small finite values (the products are discarded)
    for (uint32_t i = tid; i < (kProbeA + kProbeB) / 4; i += blockDim.x)
        reinterpret_cast<uint32_t*>(sm)[i] = tcu::to_tf32(1.0f / 1024.0f);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tcu::smem_u32(tslot)),
                     "r"(kProbeN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tcu::smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const uint64_t ad = tcu::smem_desc(tcu::smem_u32(sA), (128 / 8) * 128, 128);
        const uint64_t bd = tcu::smem_desc(tcu::smem_u32(sB), (kProbeN / 8) * 128, 128);
        for (int i = 0; i < iters; ++i) {
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(kProbeIdesc), "r"(i));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         tcu::smem_u32(mbar))
                     : "memory");
    }
    uint32_t done = 0;
    for (long long it = 0; it < tcu::kWaitLimit && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(tcu::smem_u32(mbar)), "r"(0u)
            : "memory");
    }
    if (!done && tid == 0) atomicExch(status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kProbeN));
}

}  // namespace

int peak_probe(int kind, double* out_tflops, cudaStream_t s) {
    int dev = 0, nsm = 0;
    PMLBIE_CUDA_TRY(cudaGetDevice(&dev));
    PMLBIE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    void* scratch = nullptr;
    PMLBIE_CUDA_TRY(cudaMalloc(&scratch, 4096));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double flops = 0.0;
    float ms = 0.f;
    auto launch = [&](bool timed) -> cudaError_t {
        if (timed && (e = cudaEventRecord(e0, s)) != cudaSuccess) return e;
        if (kind == 0) {
            const int iters = 4096, blocks = nsm * 8;
            fma_probe_kernel<double><<<blocks, 256, 0, s>>>(iters, 1.0, static_cast<double*>(scratch));
            flops = 2.0 * kChains * (double)iters * blocks * 256;
        } else if (kind == 1) {
            const int iters = 65536, blocks = nsm * 8;
            fma_probe_kernel<float><<<blocks, 256, 0, s>>>(iters, 1.0f, static_cast<float*>(scratch));
            flops = 2.0 * kChains * (double)iters * blocks * 256;
        } else {
            const int iters = 20000;
            tf32_probe_kernel<<<nsm, 128, kProbeSmemLaunch, s>>>(iters, static_cast<int*>(scratch));
            flops = 2.0 * 128.0 * kProbeN * 8.0 * (double)iters * nsm;
        }
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (timed && (e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
        return cudaSuccess;
    };
    if (e == cudaSuccess && kind == 2) e = cudaFuncSetAttribute(tf32_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                               (int)kProbeSmemLaunch);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, 4096, s);
    if (e == cudaSuccess) e = launch(false);
    if (e == cudaSuccess) e = launch(true);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&status, scratch, sizeof(int), cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(scratch);
    if (e != cudaSuccess) return fail(PMLBIE_ECUDA, std::string("peak probe: ") + cudaGetErrorString(e));
    if (kind == 2 && status) return fail(PMLBIE_ETIMEOUT, "peak probe: tensor-core wait expired");
    *out_tflops = flops / (ms * 1e-3) / 1e12;
    return PMLBIE_OK;
}

}  // namespace pmlbie
