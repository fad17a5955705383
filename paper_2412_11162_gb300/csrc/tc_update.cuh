// Trailing update of the FP32 LU on the 5th-generation tensor cores (sm_103a):
//
//   A22 <- A22 - L21 U12,   complex64, column-major, leading dimension n,
//
// L21 = A[k0+kb : n, k0 : k0+kb], U12 = A[k0 : k0+kb, k0+kb : n], kb <= 32.
// In 64 x 64 complex tiles of A22, the complex product is one real GEMM of
// depth 64 with the complex rows split into interleaved real rows:
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
// Per step, the split operands are formed once per 64-row block of L21
// (operand_image_kernel) and once per 64-column block of U12 (by the LU's
// block-row solve, which holds U12 in shared memory) in the exact
// shared-memory image the MMAs read: the canonical K-major layout without
// swizzling (8-row x 16-byte core matrices), hi then lo (A': 64 KB, B': 32 KB
// per block).  update_kernel (persistent, one CTA per SM, warp-specialised;
// its comment below) streams the trailing matrix through shared memory in
// 64 x 64 tiles with TMA, fetches the images with bulk copies, runs the 24
// tcgen05.mma (M = 128, N = 64, K = 8) of a tile into one of two
// tensor-memory accumulators, and subtracts the accumulator from the tile
// before a TMA store.  Rows and columns beyond n in a ragged block give
// accumulator rows / columns that are never stored (the tensor store clips
// at n).  On a wait that expires the MMAs may still be in flight when the CTA
// frees its tensor memory, so a later CTA that allocates those columns could
// see their writes: the error is reported (info[b] = -1, the solve returns
// PMLBIE_ETIMEOUT), and the factorisation's results are not used after it.
#pragma once

#include <cuda.h>

#include <cstdint>

#include "tcgen05_util.cuh"

namespace pmlbie {
namespace tcu {

constexpr int kTileC = 64;        // complex rows and columns per tile
constexpr int kRows = 128;        // real rows of A' (M of the MMA)
constexpr int kCols = 64;         // columns of B' (N of the MMA)
constexpr int kDepth = 64;        // real depth (2 x panel width 32)
constexpr uint32_t kABytes = kRows * kDepth * 4;   // 32 KB per A' copy
constexpr uint32_t kBBytes = kCols * kDepth * 4;   // 16 KB per B' copy

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

// A' operand images of one step.  Grid (nblk, 2, batch), 256 threads: y = 0,
// 1 form the first / second half of the A' image of row block x (real rows
// 0-63 / 64-127 of the 16-byte core-matrix rows).  Image byte 16 u holds real
// row r = 8 g + r8 at depths 4 kc .. 4 kc + 3, with (kc, g, r8) the digits of
// u: u = (kc R/8 + g) 8 + r8, R = 128 rows -- the layout whose K-adjacent core
// matrices are R/8 x 128 bytes apart and row-adjacent ones 128 bytes apart.
// Rows beyond n are zero-filled.  The image of mode b, block x starts at
// Aimg + (b nblk + x) kAImg.  (The B' images -- R = 64 columns, depth k < 32
// Re U[k][j], k >= 32 Im U[k-32][j], u = kc 64 + j -- are written by the LU's
// block-row solve, which holds U12 in shared memory, at Bimg + (b nblk + x) kBImg.)
__global__ void __launch_bounds__(256) operand_image_kernel(int n, int k0, int kb, int nblk, const float2* A,
                                                            unsigned char* Aimg) {
    const int b = blockIdx.z, blk = blockIdx.x;
    const float2* a = A + (size_t)b * n * n;
    const int base = k0 + kb + blk * kTileC;
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
            v[t][e] = (kk + e < kb && base + i < n) ? a[(size_t)(k0 + kk + e) * n + base + i] : make_float2(0.f, 0.f);
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

// ---------------------------------------------------------------------------
// Persistent, warp-specialised update.  One CTA per SM (224 KB of shared
// memory) walks whole rows of tiles: row units u = b nblk + bx (mode b, row
// block bx) are dealt round-robin (CTA c takes u = c, c + G, ..), so that the
// CTAs running at the same time work on neighbouring modes whose operand
// images stay in L2, and a unit's A' image is fetched once for its nblk tiles.
// Warp 0 (one thread) is the producer: the unit's A' image (bulk copy), then
// per tile the B' image (bulk copy, two stages) and the 64 x 64 A22 tile (TMA
// tensor load, three stages; rows / columns beyond n read as zeros).  Warp 1
// (one thread) issues the tile's 24 MMAs into one of two tensor-memory
// accumulators.  Warps 2-5 read the accumulator (each its lane quadrant),
// subtract it from the tile in shared memory and store the tile with a TMA
// tensor store (clipped at n).  Stages pass between the roles through
// mbarriers: full (transaction bytes / MMA commit) and empty (MMA commit,
// epilogue arrival, or the store's completed read).  Every wait is bounded; on
// expiry the CTA records the error, stops its loops (the epilogue warps decide
// together through a barrier reduction, so none waits alone), waits (bounded)
// for the copies it issued, and marks info[b] = -1 for the modes of its tiles.
constexpr int kPipeThreads = 192;            // warp 0 producer, warp 1 MMA, warps 2-5 epilogue
constexpr int kBStages = 2, kCStages = 3;
constexpr uint32_t kCTile = kTileC * kTileC * 8;                    // 32 KB complex64 tile
constexpr uint32_t kPipeOffB = kAImg;                               // after the A' image (64 KB)
constexpr uint32_t kPipeOffC = kPipeOffB + kBStages * kBImg;        // 128 KB
constexpr uint32_t kPipeOffBar = kPipeOffC + kCStages * kCTile;     // 224 KB
constexpr uint32_t kPipeSmem = kPipeOffBar + 256;
constexpr int kPipeTmemCols = 128;           // two 64-column accumulators

struct PipeBars {
    uint64_t a_full, a_empty, b_full[kBStages], b_empty[kBStages], c_full[kCStages], c_empty[kCStages],
        acc_full[2], acc_empty[2];
    uint32_t tmem;
    int err;
};
static_assert(sizeof(PipeBars) <= 256, "barrier block");

__device__ __forceinline__ void mb_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mb_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
                 : "memory");
}
// 64 x 64 tile of the [batch][n][n] complex64 tensor (8-byte elements): x = row, y = column, z = mode
__device__ __forceinline__ void tma_load_tile(uint32_t dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(b))
        : "memory");
}
__device__ __forceinline__ void tma_store_tile(const CUtensorMap* tm, int x, int y, int z, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(x), "r"(y), "r"(z), "r"(src)
                 : "memory");
}
__device__ __forceinline__ bool err_set(const PipeBars* bar) { return *reinterpret_cast<const volatile int*>(&bar->err); }

__global__ void __launch_bounds__(kPipeThreads, 1) update_kernel(const __grid_constant__ CUtensorMap tmA, int k0, int kb,
                                                                 int nblk, int batch, const unsigned char* Aimg,
                                                                 const unsigned char* Bimg, int* info) {
    extern __shared__ __align__(1024) unsigned char sm[];
    PipeBars* bar = reinterpret_cast<PipeBars*>(sm + kPipeOffBar);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long U = (long long)batch * nblk;          // row units (mode, row block)
    const long long G = gridDim.x;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bar->tmem)),
                     "r"(kPipeTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mb_init(&bar->a_full, 1);
        mb_init(&bar->a_empty, 1);
        for (int s = 0; s < kBStages; ++s) {
            mb_init(&bar->b_full[s], 1);
            mb_init(&bar->b_empty[s], 1);
        }
        for (int s = 0; s < kCStages; ++s) {
            mb_init(&bar->c_full[s], 1);
            mb_init(&bar->c_empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mb_init(&bar->acc_full[s], 1);
            mb_init(&bar->acc_empty[s], 4);   // one arrival per epilogue warp
        }
        bar->err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = bar->tmem;
    const uint32_t sbase = smem_u32(sm);
    const int rbase = k0 + kb;                            // first row / column of A22

    if (warp == 0) {
        if (lane == 0) {
            // producer
            long long i = 0, lastB[kBStages], lastC[kCStages];
            int k = 0, a_issued = 0;
            for (int s = 0; s < kBStages; ++s) lastB[s] = -1;
            for (int s = 0; s < kCStages; ++s) lastC[s] = -1;
            bool ok = true;
            for (long long u = blockIdx.x; u < U && ok; u += G, ++k) {
                const int b = (int)(u / nblk), bx = (int)(u - (long long)b * nblk);
                if (k >= 1 && !mbar_wait(smem_u32(&bar->a_empty), (uint32_t)((k - 1) & 1))) {
                    ok = false;
                    break;
                }
                mb_expect(&bar->a_full, kAImg);
                bulk_load(sbase, Aimg + (size_t)u * kAImg, kAImg, smem_u32(&bar->a_full));
                ++a_issued;
                for (int by = 0; by < nblk; ++by, ++i) {
                    const int bs = (int)(i % kBStages), cs = (int)(i % kCStages);
                    if (i >= kBStages &&
                        !mbar_wait(smem_u32(&bar->b_empty[bs]), (uint32_t)(((i / kBStages) - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    mb_expect(&bar->b_full[bs], kBImg);
                    bulk_load(sbase + kPipeOffB + bs * kBImg, Bimg + ((size_t)b * nblk + by) * kBImg, kBImg,
                              smem_u32(&bar->b_full[bs]));
                    lastB[bs] = i;
                    if (i >= kCStages &&
                        !mbar_wait(smem_u32(&bar->c_empty[cs]), (uint32_t)(((i / kCStages) - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    mb_expect(&bar->c_full[cs], kCTile);
                    tma_load_tile(sbase + kPipeOffC + cs * kCTile, &tmA, rbase + bx * kTileC, rbase + by * kTileC, b,
                                  &bar->c_full[cs]);
                    lastC[cs] = i;
                }
            }
            if (!ok) {
                bar->err = 1;
                // copies in flight: wait (bounded) for the last issued use of every stage
                if (a_issued > 0) mbar_wait(smem_u32(&bar->a_full), (uint32_t)((a_issued - 1) & 1));
                for (int s = 0; s < kBStages; ++s)
                    if (lastB[s] >= 0) mbar_wait(smem_u32(&bar->b_full[s]), (uint32_t)((lastB[s] / kBStages) & 1));
                for (int s = 0; s < kCStages; ++s)
                    if (lastC[s] >= 0) mbar_wait(smem_u32(&bar->c_full[s]), (uint32_t)((lastC[s] / kCStages) & 1));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issue: hi*hi, hi*lo, lo*hi; each K = 8 step covers two K-adjacent core matrices
            const uint32_t aLBO = (kRows / 8) * 128, bLBO = (kCols / 8) * 128, SBO = 128;
            long long i = 0;
            int k = 0;
            bool ok = true;
            for (long long u = blockIdx.x; u < U && ok; u += G, ++k) {
                if (err_set(bar) || !mbar_wait(smem_u32(&bar->a_full), (uint32_t)(k & 1))) {
                    ok = false;
                    break;
                }
                for (int by = 0; by < nblk; ++by, ++i) {
                    const int bs = (int)(i % kBStages), ab = (int)(i & 1);
                    if (err_set(bar) || !mbar_wait(smem_u32(&bar->b_full[bs]), (uint32_t)((i / kBStages) & 1)) ||
                        (i >= 2 && !mbar_wait(smem_u32(&bar->acc_empty[ab]), (uint32_t)(((i >> 1) - 1) & 1)))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t ah = sbase, al = sbase + kABytes;
                    const uint32_t bh = sbase + kPipeOffB + bs * kBImg, bl = bh + kBBytes;
                    const uint32_t d = tmem + (uint32_t)(ab * kTileC);
#pragma unroll
                    for (int pass = 0; pass < 3; ++pass) {
                        const uint32_t sa = pass == 2 ? al : ah, sb = pass == 1 ? bl : bh;
#pragma unroll
                        for (int s = 0; s < kDepth / 8; ++s) {
                            const uint64_t ad = smem_desc(sa + s * 2 * aLBO, aLBO, SBO);
                            const uint64_t bd = smem_desc(sb + s * 2 * bLBO, bLBO, SBO);
                            mma_tf32(d, ad, bd, (pass | s) != 0);
                        }
                    }
                    mma_commit(&bar->b_empty[bs]);
                    mma_commit(&bar->acc_full[ab]);
                    if (by == nblk - 1) mma_commit(&bar->a_empty);
                }
            }
            if (!ok) bar->err = 1;
        }
    } else {
        // epilogue: this warp's lane quadrant of the accumulator (real rows 32 q ..)
        const int q = warp & 3;
        const int rr = 32 * q + lane, row = rr >> 1, part = rr & 1;
        const bool leader = tid == 64;
        long long i = 0;
        bool stop = false;
        for (long long u = blockIdx.x; u < U && !stop; u += G) {
            const int b = (int)(u / nblk), bx = (int)(u - (long long)b * nblk);
            for (int by = 0; by < nblk; ++by, ++i) {
                const int ab = (int)(i & 1), cs = (int)(i % kCStages);
                const bool ok = mbar_wait(smem_u32(&bar->acc_full[ab]), (uint32_t)((i >> 1) & 1)) &&
                                mbar_wait(smem_u32(&bar->c_full[cs]), (uint32_t)((i / kCStages) & 1));
                if (!ok) bar->err = 1;
                // one decision for all 128 epilogue threads (a barrier with an OR
                // reduction), so that none of them waits at a later barrier alone
                uint32_t any;
                asm volatile(
                    "{\n\t.reg .pred p, q;\n\t"
                    "setp.ne.u32 p, %1, 0;\n\t"
                    "bar.red.or.pred q, 1, 128, p;\n\t"
                    "selp.u32 %0, 1, 0, q;\n\t}\n"
                    : "=r"(any)
                    : "r"((uint32_t)(!ok || err_set(bar)))
                    : "memory");
                if (any) {
                    stop = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // tile element (column c, row) at 8 (64 c + row) bytes; this thread's real part or imaginary part
                float* ct = reinterpret_cast<float*>(sm + kPipeOffC + cs * kCTile) + 2 * row + part;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float pv[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * kTileC + 32 * h), pv);
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        float* e = ct + (size_t)(32 * h + c) * 2 * kTileC;
                        *e = *e - pv[c];
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mb_arrive(&bar->acc_empty[ab]);
                // generic-proxy tile writes -> visible to the TMA store
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (leader) {
                    tma_store_tile(&tmA, rbase + bx * kTileC, rbase + by * kTileC, b, sbase + kPipeOffC + cs * kCTile);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    // the previous tile's store has read its buffer: release that stage
                    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                    if (i >= 1) mb_arrive(&bar->c_empty[(int)((i - 1) % kCStages)]);
                }
            }
        }
        if (leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (err_set(bar) && tid == 0)
        for (long long u = blockIdx.x; u < U; u += G) info[u / nblk] = -1;
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPipeTmemCols));
}

}  // namespace tcu
}  // namespace pmlbie
