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
// Two launches per step.  operand_image_kernel forms, once per 64-row block of
// L21 and once per 64-column block of U12, the split operands in the exact
// shared-memory image the MMAs read: the canonical K-major layout without
// swizzling (8-row x 16-byte core matrices), hi then lo (A': 64 KB, B': 32 KB
// per block).  update_kernel then fetches its tile's two images with two bulk
// copies (cp.async.bulk, completion counted in bytes on an mbarrier) while its
// threads load their A22 values, so no CTA re-reads or re-splits operands; one
// thread issues the 24 tcgen05.mma (M = 128, N = 64, K = 8), completion is
// signalled through a second mbarrier (tcgen05.commit), and the epilogue reads
// the accumulator with tcgen05.ld (warp w: lanes 32 (w mod 4) .., columns
// 32 (w / 4) ..) and subtracts it from A22 in place.  Rows and columns beyond
// n in a ragged block give accumulator rows / columns that are never stored.
// Every mbarrier wait is bounded: on expiry the CTA records info[b] = -1 and
// skips its epilogue (the solve then returns PMLBIE_ETIMEOUT); a CTA whose
// operand copies did not arrive waits for them once more (bounded) before it
// exits.  On a real expiry the MMAs may still be in flight when the CTA frees
// its tensor memory, so a later CTA that allocates those columns could see
// their writes: the error is reported, and the factorisation's results are
// not used after it.
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
// the allocation whichever way the two byte offsets are read), then the two
// mbarriers (images arrived, MMAs done), the tensor-memory address and a flag
constexpr uint32_t kSlack = 8192;
constexpr uint32_t kSmemBytes = 2 * kABytes + 2 * kBBytes + kSlack + 64;

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

// bytes of one block's operand images (hi then lo)
constexpr uint32_t kAImg = 2 * kABytes;
constexpr uint32_t kBImg = 2 * kBBytes;

// 64-row / 64-column blocks of the trailing matrix at step k0 (kb = 32)
__host__ __device__ constexpr int update_blocks(int n, int k0, int kb) { return (n - k0 - kb + kTileC - 1) / kTileC; }

// Operand images of one step.  Grid (nblk, 3, batch), 256 threads: y = 0, 1
// form the first / second half of the A' image of row block x (real rows
// 0-63 / 64-127 of the 16-byte core-matrix rows), y = 2 the B' image of column
// block x.  Image byte 16 u holds real row (or column) r = 8 g + r8 at depths
// 4 kc .. 4 kc + 3, with (kc, g, r8) the digits of u: u = (kc R/8 + g) 8 + r8,
// R = 128 rows for A', 64 columns for B' -- the layout whose K-adjacent core
// matrices are R/8 x 128 bytes apart and row-adjacent ones 128 bytes apart.
// Rows and columns beyond n are zero-filled.  Images of mode b, block x start
// at Aimg + (b nblk + x) kAImg and Bimg + (b nblk + x) kBImg.
__global__ void __launch_bounds__(256) operand_image_kernel(int n, int k0, int kb, int nblk, const float2* A,
                                                            unsigned char* Aimg, unsigned char* Bimg) {
    const int b = blockIdx.z, blk = blockIdx.x;
    const float2* a = A + (size_t)b * n * n;
    const int base = k0 + kb + blk * kTileC;
    if (blockIdx.y < 2) {
        uint4* hi = reinterpret_cast<uint4*>(Aimg + ((size_t)b * nblk + blk) * kAImg);
        uint4* lo = hi + kABytes / 16;
        constexpr int kIt = kABytes / 16 / 2 / 256;   // 4 core-matrix rows per thread
        float2 v[kIt][4];
#pragma unroll
        for (int t = 0; t < kIt; ++t) {
            // half y covers core-matrix groups g = 8 y .. 8 y + 7 of every kc
            const int w = threadIdx.x + t * 256;           // 0 .. 1023
            const int kc = w >> 6, g = ((w >> 3) & 7) + 8 * blockIdx.y, r8 = w & 7;
            const int i = (g * 8 + r8) >> 1, kk = (kc * 4) & 31;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                v[t][e] = (kk + e < kb && base + i < n) ? a[(size_t)(k0 + kk + e) * n + base + i]
                                                        : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < kIt; ++t) {
            const int w = threadIdx.x + t * 256;
            const int kc = w >> 6, g = ((w >> 3) & 7) + 8 * blockIdx.y, r8 = w & 7;
            const int part = r8 & 1, u = (kc * 16 + g) * 8 + r8;
            // depths 0-31 multiply Re U, 32-63 Im U: row 2i = (Re L, -Im L), row 2i+1 = (Im L, Re L)
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float x = kc < 8 ? (part ? v[t][e].y : v[t][e].x) : (part ? v[t][e].x : -v[t][e].y);
                split_tf32(x, h[e], l[e]);
            }
            hi[u] = make_uint4(h[0], h[1], h[2], h[3]);
            lo[u] = make_uint4(l[0], l[1], l[2], l[3]);
        }
    } else {
        uint4* hi = reinterpret_cast<uint4*>(Bimg + ((size_t)b * nblk + blk) * kBImg);
        uint4* lo = hi + kBBytes / 16;
        constexpr int kIt = kBBytes / 16 / 256;       // 4
        float2 v[kIt][4];
#pragma unroll
        for (int t = 0; t < kIt; ++t) {
            const int u = threadIdx.x + t * 256;
            const int kc = u >> 6, j = u & 63, kk = (kc * 4) & 31;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                v[t][e] = (kk + e < kb && base + j < n) ? a[(size_t)(base + j) * n + k0 + kk + e]
                                                        : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < kIt; ++t) {
            const int u = threadIdx.x + t * 256, kc = u >> 6;
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) split_tf32(kc < 8 ? v[t][e].x : v[t][e].y, h[e], l[e]);
            hi[u] = make_uint4(h[0], h[1], h[2], h[3]);
            lo[u] = make_uint4(l[0], l[1], l[2], l[3]);
        }
    }
}

// bounded wait on phase `parity` of an mbarrier; false on expiry
__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity) {
    uint32_t done = 0;
    for (long long it = 0; it < kWaitLimit && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mb), "r"(parity)
            : "memory");
    }
    return done != 0;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mb) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mb)
                 : "memory");
}

__global__ void __launch_bounds__(kThreads, 2) update_kernel(int n, int k0, int kb, int nblk, float2* A,
                                                             const unsigned char* Aimg, const unsigned char* Bimg,
                                                             int* info) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* sAhi = sm;
    unsigned char* sAlo = sAhi + kABytes;
    unsigned char* sBhi = sAlo + kABytes;
    unsigned char* sBlo = sBhi + kBBytes;
    unsigned char* tail = sBlo + kBBytes + kSlack;
    uint64_t* mb_ld = reinterpret_cast<uint64_t*>(tail);
    uint64_t* mb_mma = reinterpret_cast<uint64_t*>(tail + 8);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tail + 16);
    int* flag = reinterpret_cast<int*>(tail + 20);

    const int b = blockIdx.z;
    float2* a = A + (size_t)b * n * n;
    const int r0 = k0 + kb + blockIdx.x * kTileC, c0 = k0 + kb + blockIdx.y * kTileC;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kIssuer = 32;   // first thread of warp 1 (warp 0 allocates tensor memory meanwhile)

    // tensor memory for the 128 x 64 FP32 accumulator (warp 0 allocates)
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == kIssuer) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mb_ld)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mb_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *flag = 0;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mb_ld)),
                     "r"(kAImg + kBImg)
                     : "memory");
        bulk_load(smem_u32(sAhi), Aimg + ((size_t)b * nblk + blockIdx.x) * kAImg, kAImg, smem_u32(mb_ld));
        bulk_load(smem_u32(sBhi), Bimg + ((size_t)b * nblk + blockIdx.y) * kBImg, kBImg, smem_u32(mb_ld));
    }

    // this thread's 32 values of A22 (the DRAM traffic), loaded while the images arrive
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
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (tid == kIssuer) {
        if (mbar_wait(smem_u32(mb_ld), 0)) {
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
                             smem_u32(mb_mma))
                         : "memory");
        } else {
            // the images did not arrive: record it, release the other threads,
            // and wait once more (bounded) for the copies before exiting
            *flag = 1;
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mb_mma)) : "memory");
            mbar_wait(smem_u32(mb_ld), 0);
        }
    }
    if (!mbar_wait(smem_u32(mb_mma), 0)) *flag = 1;
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
