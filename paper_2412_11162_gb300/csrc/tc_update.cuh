// Trailing update of the FP32 LU on the 5th-generation tensor cores (sm_103a):
//
//   A22 <- A22 - L21 U12,   complex64, column-major, leading dimension n,
//
// L21 = A[k0+kb : n, k0 : k0+kb], U12 = A[k0 : k0+kb, k0+kb : n], kb <= 32.
// One CTA per 64 x 64 complex tile of A22.  The complex product is one real
// GEMM of depth 64 with the complex rows split into interleaved real rows:
//
//   P[2i  ][j] = sum_k  Re L[i][k] Re U[k][j] - Im L[i][k] Im U[k][j]
//   P[2i+1][j] = sum_k  Im L[i][k] Re U[k][j] + Re L[i][k] Im U[k][j]
//
// i.e. A' = [[Re L, -Im L] ; [Im L, Re L]] row-interleaved (128 x 64) and
// B' = [Re U ; Im U] (64 x 64).  FP32 accuracy from TF32 inputs by the split
// x = hi + lo (hi = TF32 rounding of x, lo = TF32 rounding of x - hi):
// P ~ A'hi B'hi + A'hi B'lo + A'lo B'hi, accumulated in FP32 in tensor memory
// (relative error ~1e-6 of |L||U|, i.e. FP32 level: the LU stays a
// preconditioner for the FP64 refinement).
//
// Operands are staged by the CTA's threads from global memory into shared
// memory in the canonical K-major layout without swizzling (8-row x 16-byte
// core matrices), 24 tcgen05.mma (M = 128, N = 64, K = 8) are issued by one
// thread, completion is signalled through an mbarrier (tcgen05.commit), and the
// epilogue reads the accumulator with tcgen05.ld (warp w: lanes 32 (w mod 4) ..,
// columns 32 (w / 4) ..) and subtracts it from A22 in place; the A22 values are
// loaded together with the operands, before the MMAs.  The mbarrier wait is bounded: on expiry the CTA
// records info[b] = -1 and skips its epilogue (the solve then returns PMLBIE_ETIMEOUT).  On a real
// expiry the MMAs may still be in flight when the CTA frees its tensor memory, so a later CTA that
// allocates those columns could see their writes: the error is reported, and the factorisation's
// results are not used after it.
#pragma once

#include <cstdint>

#include "tcgen05_util.cuh"

namespace pmlbie {
namespace tcu {

constexpr int kTileC = 64;        // complex rows and columns per CTA
constexpr int kRows = 128;        // real rows of A' (M of the MMA)
constexpr int kCols = 64;         // columns of B' (N of the MMA)
constexpr int kDepth = 64;        // real depth (2 x panel width 32)
constexpr int kThreads = 256;
constexpr int kTmemCols = 64;
constexpr uint32_t kABytes = kRows * kDepth * 4;   // 32 KB per A' copy
constexpr uint32_t kBBytes = kCols * kDepth * 4;   // 16 KB per B' copy
// operands, then 8 KB of slack (every descriptor-addressed byte stays inside
// the allocation whichever way the two byte offsets are read), then the
// mbarrier, the tensor-memory address and a flag
constexpr uint32_t kSlack = 8192;
constexpr uint32_t kSmemBytes = 2 * kABytes + 2 * kBBytes + kSlack + 64;

// Byte offset of element (r, k) of a K-major operand with R rows: core matrix
// (k / 4, r / 8) of 128 bytes, K-adjacent core matrices R/8 * 128 bytes apart
// (leading byte offset), row-adjacent ones 128 bytes apart (stride byte offset).
__device__ __forceinline__ uint32_t core_off(int r, int k, int R) {
    return (uint32_t)((((k >> 2) * (R >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 3) << 2));
}

// Instruction descriptor, kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kCols >> 3) << 17) |
                            ((uint32_t)(kRows >> 4) << 24);

// x -> (hi, lo) TF32 pair stored as 32-bit containers
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}

__global__ void __launch_bounds__(kThreads, 2) update_kernel(int n, int k0, int kb, float2* A, int* info) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* sAhi = sm;
    unsigned char* sAlo = sAhi + kABytes;
    unsigned char* sBhi = sAlo + kABytes;
    unsigned char* sBlo = sBhi + kBBytes;
    unsigned char* tail = sBlo + kBBytes + kSlack;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(tail);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tail + 8);
    int* flag = reinterpret_cast<int*>(tail + 16);

    const int b = blockIdx.z;
    float2* a = A + (size_t)b * n * n;
    const int r0 = k0 + kb + blockIdx.x * kTileC, c0 = k0 + kb + blockIdx.y * kTileC;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // tensor memory for the 128 x 64 FP32 accumulator (warp 0 allocates)
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *flag = 0;
    }

    // All global loads of the CTA are issued before any of them is used: this
    // thread's 32 values of A22 first (the DRAM traffic), then the A' and B'
    // elements (8 + 8 per thread, mostly served by L2).
    const int q = warp & 3, h = warp >> 2;
    const int rr = 32 * q + lane;                 // real row of P
    const int row = r0 + (rr >> 1), part = rr & 1;
    const int cbase = c0 + 32 * h;
    // columns by one pointer stepped by the column stride (2n floats)
    float* pc = reinterpret_cast<float*>(a) + 2 * ((size_t)cbase * n + row) + part;
    const size_t cstride = 2 * (size_t)n;
    const int ncv = row < n ? min(32, n - cbase) : 0;
    float cv[32];
    {
        const float* p = pc;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            cv[c] = c < ncv ? *p : 0.f;
            p += cstride;
        }
    }
    constexpr int kPer = kTileC * 32 / kThreads;   // 8
    float2 lv[kPer], uv[kPer];
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
        // A' from L21: element (i, k) of L -> rows 2i, 2i+1 at depths k, 32+k;
        // this (i, k) order keeps each warp's shared stores on 16 banks
        const int e = tid + t * kThreads;
        const int i = (e & 3) | (((e >> 4) & 1) << 2) | (((e >> 5) & 7) << 3);
        const int k = ((e >> 2) & 3) | ((e >> 8) << 2);
        lv[t] = (k < kb && r0 + i < n) ? a[(size_t)(k0 + k) * n + r0 + i] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
        // B' from U12: element (k, j) of U -> column j at depths k (Re), 32+k (Im)
        const int e = tid + t * kThreads;
        const int k = (e & 3) | (((e >> 5) & 7) << 2);
        const int j = ((e >> 2) & 7) | ((e >> 8) << 3);
        uv[t] = (k < kb && c0 + j < n) ? a[(size_t)(c0 + j) * n + k0 + k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
        const int e = tid + t * kThreads;
        const int i = (e & 3) | (((e >> 4) & 1) << 2) | (((e >> 5) & 7) << 3);
        const int k = ((e >> 2) & 3) | ((e >> 8) << 2);
        uint32_t reh, rel, imh, iml, nih, nil;
        split_tf32(lv[t].x, reh, rel);
        split_tf32(lv[t].y, imh, iml);
        split_tf32(-lv[t].y, nih, nil);
        const uint32_t o00 = core_off(2 * i, k, kRows), o01 = core_off(2 * i, 32 + k, kRows);
        const uint32_t o10 = core_off(2 * i + 1, k, kRows), o11 = core_off(2 * i + 1, 32 + k, kRows);
        *reinterpret_cast<uint32_t*>(sAhi + o00) = reh;
        *reinterpret_cast<uint32_t*>(sAlo + o00) = rel;
        *reinterpret_cast<uint32_t*>(sAhi + o01) = nih;
        *reinterpret_cast<uint32_t*>(sAlo + o01) = nil;
        *reinterpret_cast<uint32_t*>(sAhi + o10) = imh;
        *reinterpret_cast<uint32_t*>(sAlo + o10) = iml;
        *reinterpret_cast<uint32_t*>(sAhi + o11) = reh;
        *reinterpret_cast<uint32_t*>(sAlo + o11) = rel;
    }
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
        const int e = tid + t * kThreads;
        const int k = (e & 3) | (((e >> 5) & 7) << 2);
        const int j = ((e >> 2) & 7) | ((e >> 8) << 3);
        uint32_t reh, rel, imh, iml;
        split_tf32(uv[t].x, reh, rel);
        split_tf32(uv[t].y, imh, iml);
        const uint32_t o0 = core_off(j, k, kCols), o1 = core_off(j, 32 + k, kCols);
        *reinterpret_cast<uint32_t*>(sBhi + o0) = reh;
        *reinterpret_cast<uint32_t*>(sBlo + o0) = rel;
        *reinterpret_cast<uint32_t*>(sBhi + o1) = imh;
        *reinterpret_cast<uint32_t*>(sBlo + o1) = iml;
    }
    // generic-proxy shared stores -> visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (tid == 0) {
        const uint32_t aLBO = (kRows / 8) * 128, bLBO = (kCols / 8) * 128, SBO = 128;
        const uint32_t ah = smem_u32(sAhi), al = smem_u32(sAlo), bh = smem_u32(sBhi), bl = smem_u32(sBlo);
        // hi*hi, hi*lo, lo*hi; each K = 8 step covers two K-adjacent core matrices
#pragma unroll
        for (int pass = 0; pass < 3; ++pass) {
            const uint32_t sa = pass == 2 ? al : ah, sb = pass == 1 ? bl : bh;
#pragma unroll
            for (int s = 0; s < kDepth / 8; ++s) {
                const uint64_t ad = smem_desc(sa + s * 2 * aLBO, aLBO, SBO);
                const uint64_t bd = smem_desc(sb + s * 2 * bLBO, bLBO, SBO);
                mma_tf32(tmem, ad, bd, (pass | s) != 0);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(mbar))
                     : "memory");
    }

    // bounded wait for the MMAs (phase 0)
    uint32_t done = 0;
    for (long long it = 0; it < kWaitLimit && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(0u)
            : "memory");
    }
    if (!done) *flag = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (*flag == 0) {
        float pv[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * h), pv);
        float* p = pc;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            if (c < ncv) *p = cv[c] - pv[c];
            p += cstride;
        }
    } else if (tid == 0) {
        info[b] = -1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace tcu
}  // namespace pmlbie
