// Batched dense complex LU with partial pivoting (one matrix per Fourier
// mode), triangular solves, and the FP64 residual / FP32 correction steps of
// mixed-precision iterative refinement.
//
// The per-mode systems are the transmission block systems of Wang & Lu,
// arXiv 2412.11162, Sec. 4.2 (Eqs. (ntdpsi1), (ntdpsi2) in block form); the
// factorisation itself is textbook right-looking blocked LU: panel
// factorisation (pivot search, row swap, scaling, rank-1 updates inside the
// panel), row swaps + unit-lower triangular solve for the block row, and a
// tiled GEMM update of the trailing matrix (complex128: FP64 CUDA cores;
// complex64: tcgen05 tensor cores on split operand images formed once per
// step, tc_update.cuh).  complex128 leaves LAPACK getrf's row order (every
// column swapped) and a row permutation in piv; complex64 swaps only the
// columns right of each panel, so L's column blocks keep their step's row
// order, and the solves apply each step's interchanges (the per-step slot
// mapping in ptab) when they reach the step's block -- the same forward
// substitution.  Matrices are column-major, A[b][col][row], leading
// dimension n.  info[b] > 0 marks the first zero pivot, info[b] = -1 a
// tensor-core update that did not complete.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <utility>

#include <cudaTypedefs.h>

#include "internal.h"
#include "tc_update.cuh"

namespace pmlbie {

namespace {

template <typename T> struct Cx;
template <> struct Cx<double2> {
    using R = double;
    static __device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }
};
template <> struct Cx<float2> {
    using R = float;
    static __device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
};

template <typename T> __device__ __forceinline__ T add(T a, T b) { return Cx<T>::mk(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ T sub(T a, T b) { return Cx<T>::mk(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ T mul(T a, T b) {
    return Cx<T>::mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a - b*c
template <typename T> __device__ __forceinline__ T fms(T a, T b, T c) {
    return Cx<T>::mk(a.x - b.x * c.x + b.y * c.y, a.y - b.x * c.y - b.y * c.x);
}
// a + b*c
template <typename T> __device__ __forceinline__ T fma_c(T a, T b, T c) {
    return Cx<T>::mk(a.x + b.x * c.x - b.y * c.y, a.y + b.x * c.y + b.y * c.x);
}
template <typename T> __device__ __forceinline__ T rcp(T a) {
    using R = typename Cx<T>::R;
    R s = fmax(fabs(a.x), fabs(a.y));
    R ax = a.x / s, ay = a.y / s, d = ax * ax + ay * ay;
    return Cx<T>::mk(ax / (d * s), -ay / (d * s));
}
template <typename T> __device__ __forceinline__ typename Cx<T>::R abs2(T a) { return a.x * a.x + a.y * a.y; }

constexpr int kNB = 32;          // panel width
constexpr int kPanelThreads = 512;

// Panel factorisation of columns [k0, k0+kb) over rows [k0, n), one CTA per
// matrix.  The panel is processed in sub-panels of w columns that are held in
// shared memory (m = n - k0 rows, m x w entries), left-looking inside the
// panel: a sub-panel is loaded, brought up to date with the sub-panels to its
// left (unit-lower solve on its top rows, then the rank-s0 update of the rows
// below, s0 = columns already factored), factored column by column in shared
// memory (pivot search, swap, scaling, rank-1 updates), and written back.
// Each row interchange is applied at once to the panel's other columns in
// global memory (the L part of the earlier sub-panels and the not yet loaded
// later ones), so the panel leaves with LAPACK getrf's row order.
template <typename T>
__global__ void __launch_bounds__(kPanelThreads) panel_kernel(int n, int k0, int kb, int w, T* A, int* piv,
                                                              int* info) {
    using R = typename Cx<T>::R;
    extern __shared__ unsigned char smraw[];
    T* S = reinterpret_cast<T*>(smraw);          // [w][m], S[c * m + i], i = row - k0
    __shared__ R sval[kPanelThreads / 32];
    __shared__ int sidx[kPanelThreads / 32];
    __shared__ int spiv;
    __shared__ T sinv;
    const int m = n - k0;
    T* a = A + (size_t)blockIdx.x * n * n;
    int* pv = piv + (size_t)blockIdx.x * n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    for (int s0 = 0; s0 < kb; s0 += w) {
        const int ws = min(w, kb - s0);
        for (int idx = tid; idx < ws * m; idx += nt) {
            const int c = idx / m, i = idx - c * m;
            S[idx] = a[(size_t)(k0 + s0 + c) * n + k0 + i];
        }
        __syncthreads();
        if (s0 > 0) {
            // top rows: U = L11^{-1} (rows 0..s0-1), one warp per column, lane = row
            for (int c = warp; c < ws; c += nt >> 5) {
                T x = lane < s0 ? S[c * m + lane] : Cx<T>::mk(0, 0);
                for (int t = 0; t < s0 - 1; ++t) {
                    const T xt = Cx<T>::mk(__shfl_sync(0xffffffffu, x.x, t), __shfl_sync(0xffffffffu, x.y, t));
                    if (lane > t && lane < s0) x = fms(x, a[(size_t)(k0 + t) * n + k0 + lane], xt);
                }
                if (lane < s0) S[c * m + lane] = x;
            }
            __syncthreads();
            // rows below: S[c][i] -= sum_t L[i][t] U[t][c], one thread per row,
            // eight columns at a time
            for (int i = s0 + tid; i < m; i += nt) {
                for (int c0 = 0; c0 < ws; c0 += 8) {
                    T acc[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[c] = Cx<T>::mk(0, 0);
#pragma unroll 4
                    for (int t = 0; t < s0; ++t) {
                        const T l = a[(size_t)(k0 + t) * n + k0 + i];
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            if (c0 + c < ws) {
                                const T u = S[(size_t)(c0 + c) * m + t];
                                acc[c].x += l.x * u.x - l.y * u.y;
                                acc[c].y += l.x * u.y + l.y * u.x;
                            }
                    }
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (c0 + c < ws) S[(size_t)(c0 + c) * m + i] = sub(S[(size_t)(c0 + c) * m + i], acc[c]);
                }
            }
            __syncthreads();
        }
        for (int jj = 0; jj < ws; ++jj) {
            const int j = s0 + jj;                 // local row of the diagonal entry
            const T* col = S + (size_t)jj * m;
            R best = -1;
            int bi = j;
            for (int i = j + tid; i < m; i += nt) {
                const R v = abs2(col[i]);
                if (v > best) {
                    best = v;
                    bi = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const R ov = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) {
                    best = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                sval[warp] = best;
                sidx[warp] = bi;
            }
            __syncthreads();
            if (warp == 0) {
                const int nw = nt >> 5;
                R b = lane < nw ? sval[lane] : (R)-2;
                int bix = lane < nw ? sidx[lane] : 0x7fffffff;
                for (int o = 16; o > 0; o >>= 1) {
                    const R ov = __shfl_down_sync(0xffffffffu, b, o);
                    const int oi = __shfl_down_sync(0xffffffffu, bix, o);
                    if (ov > b || (ov == b && oi < bix)) {
                        b = ov;
                        bix = oi;
                    }
                }
                if (lane == 0) {
                    spiv = bix;
                    pv[k0 + j] = k0 + bix;
                    const T d = col[bix];
                    if (b <= (R)0) {
                        if (info[blockIdx.x] == 0) info[blockIdx.x] = k0 + j + 1;
                        sinv = Cx<T>::mk(0, 0);
                    } else {
                        sinv = rcp(d);
                    }
                }
            }
            __syncthreads();
            const int p = spiv;
            if (p != j)
                for (int c = tid; c < kb; c += nt) {
                    if (c >= s0 && c < s0 + ws) {
                        T* sc = S + (size_t)(c - s0) * m;
                        const T t = sc[j];
                        sc[j] = sc[p];
                        sc[p] = t;
                    } else {
                        T* gc = a + (size_t)(k0 + c) * n + k0;
                        const T t = gc[j];
                        gc[j] = gc[p];
                        gc[p] = t;
                    }
                }
            __syncthreads();
            // scale column j below the diagonal, rank-1 update of the sub-panel's later columns
            const T inv = sinv;
            for (int i = j + 1 + tid; i < m; i += nt) {
                const T l = mul(S[(size_t)jj * m + i], inv);
                S[(size_t)jj * m + i] = l;
                for (int cc = jj + 1; cc < ws; ++cc)
                    S[(size_t)cc * m + i] = fms(S[(size_t)cc * m + i], l, S[(size_t)cc * m + j]);
            }
            __syncthreads();
        }
        for (int idx = tid; idx < ws * m; idx += nt) {
            const int c = idx / m, i = idx - c * m;
            a[(size_t)(k0 + s0 + c) * n + k0 + i] = S[idx];
        }
        __syncthreads();
    }
}

// Shared state of one panel_reg_kernel CTA, passed to its column steps.
template <int RPT, int W, int NT>
struct PanelCtx {
    float2* S1;
    int* perm;
    int* pv;
    int* info;
    float2 (*crow)[W];
    unsigned (*ckey)[NT / 32];
    float2* civ;
    float2 (*rowj)[W];
    int m, k0, s0, ws, sp, tid, lane, warp;
};

// Pivot candidate key of a row at position pos (< 1024) with value v: a valid
// bit, the top 21 bits of |v|^2 (exponent and 13 mantissa bits; non-negative
// floats order like their bit patterns) and 1023 - pos, so that the largest
// key is the largest |v|^2 to 13 bits, ties going to the smallest position;
// 0 = no candidate.  One warp-wide unsigned max (redux.sync) then finds the
// pivot of a warp's rows.
__device__ __forceinline__ unsigned pivot_key(float2 v, int pos) {
    return 0x80000000u | (__float_as_uint(abs2(v)) & 0x7FFFFC00u) | (unsigned)(1023 - pos);
}
__device__ __forceinline__ int key_pos(unsigned key) { return 1023 - (int)(key & 1023u); }

// 1 / d for the pivot, scaled by max(|Re d|, |Im d|) against overflow (the
// correctly rounded reciprocal: with the hardware approximation the refined
// solutions of the ill-conditioned high modes moved by a few 1e-6)
__device__ __forceinline__ float2 pivot_rcp(float2 d) {
    const float s = fmaxf(fabsf(d.x), fabsf(d.y));
    const float rs = __frcp_rn(s);
    const float ax = d.x * rs, ay = d.y * rs;
    const float t = __frcp_rn(ax * ax + ay * ay) * rs;
    return make_float2(ax * t, -ay * t);
}

// Column jj = g + JG of a sub-panel, after its register rows were rotated by g
// (columns g .. W-1 at indices 0 .. W-1-g, the finished columns 0 .. g-1 at
// W-g .. W-1): publish this warp's pivot candidate (|v|^2, position, row and
// 1 / v), one barrier, pick the pivot, exchange the two rows whole, scale and
// update, and form this thread's candidate for the next column.
template <int RPT, int W, int NT, int JG>
__device__ __forceinline__ void panel_column(float2 (&x)[RPT][W], unsigned& key, const PanelCtx<RPT, W, NT>& c,
                                             int g) {
    constexpr int NW = NT / 32;
    static_assert(NW <= 32, "one candidate per lane");
    const int jj = g + JG;
    if (jj >= c.ws) return;
    const int j = c.s0 + jj, buf = jj & 1;
    const int tid = c.tid, lane = c.lane, warp = c.warp;
    // every warp's best key, then (barrier) the pivot position p; the owner of
    // p publishes its row and 1 / pivot (barrier); the owner of the diagonal
    // position j published its row with the keys
    const unsigned wkey = __reduce_max_sync(0xffffffffu, key);
    if (lane == 0) c.ckey[buf][warp] = wkey;
    if (tid == j)
#pragma unroll
        for (int q = 0; q < W; ++q) c.rowj[buf][q] = x[0][q];
    __syncthreads();
    const unsigned gkey = __reduce_max_sync(0xffffffffu, lane < NW ? c.ckey[buf][lane] : 0u);
    const int p = key_pos(gkey);
    const bool nonzero = (gkey & 0x7FFFFC00u) != 0u;
    // slot choices as value selects: a branch per slot lets the compiler index
    // the register rows dynamically, which moves them to local memory
    if (tid == p % NT) {
        const int slot = p / NT;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            float2 v = x[0][q];
#pragma unroll
            for (int s = 1; s < RPT; ++s) v = slot == s ? x[s][q] : v;
            c.crow[buf][q] = v;
        }
        float2 d = x[0][JG];
#pragma unroll
        for (int s = 1; s < RPT; ++s) d = slot == s ? x[s][JG] : d;
        c.civ[buf] = nonzero ? pivot_rcp(d) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* prow = c.crow[buf];
    const float2 inv = c.civ[buf];
    if (tid == NT - 1) {   // the last warp: warp 0 holds the diagonal row's work
        c.pv[c.k0 + j] = c.k0 + p;
        if (!nonzero && c.info[blockIdx.x] == 0) c.info[blockIdx.x] = c.k0 + j + 1;
        const int t = c.perm[j];
        c.perm[j] = c.perm[p];
        c.perm[p] = t;
    }
    if (p != j) {
        if (tid == j)
#pragma unroll
            for (int q = 0; q < W; ++q) x[0][q] = prow[q];
        if (tid == p % NT) {
            const int slot = p / NT;
#pragma unroll
            for (int q = 0; q < W; ++q) {
                const float2 v = c.rowj[buf][q];
#pragma unroll
                for (int s = 0; s < RPT; ++s) x[s][q] = slot == s ? v : x[s][q];
            }
        }
        if constexpr (RPT > 1) {
            if (c.sp > 0 && tid < c.s0) {
                float2* col = c.S1 + (size_t)tid * c.m;
                const float2 t = col[j];
                col[j] = col[p];
                col[p] = t;
            }
        }
    }
    // scale below the diagonal, rank-1 update of the later columns (indices
    // JG+1 .. W-1-g), next candidate
    float2 l[RPT];
    bool act[RPT];
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
        const int i = s * NT + tid;
        act[s] = i > j && i < c.m;
        l[s] = make_float2(0.f, 0.f);
        if (act[s]) {
            l[s] = mul(x[s][JG], inv);
            x[s][JG] = l[s];
        }
    }
    bool any = false;
#pragma unroll
    for (int s = 0; s < RPT; ++s) any = any || act[s];
    if (__any_sync(0xffffffffu, any))
#pragma unroll
    for (int q = JG + 1; q < W; ++q) {
        if (q < W - g) {
            const float2 uq = prow[q];
#pragma unroll
            for (int s = 0; s < RPT; ++s)
                if (act[s]) x[s][q] = fms(x[s][q], l[s], uq);
        }
    }
    key = 0u;
    if constexpr (JG + 1 < W) {
        if (jj + 1 < c.ws) {
#pragma unroll
            for (int s = 0; s < RPT; ++s)
                if (act[s]) key = max(key, pivot_key(x[s][JG + 1], s * NT + tid));
        }
    }
}

template <int RPT, int W, int NT, int... JG>
__device__ __forceinline__ void panel_group(float2 (&x)[RPT][W], unsigned& key, const PanelCtx<RPT, W, NT>& c, int g,
                                            std::integer_sequence<int, JG...>) {
    (panel_column<RPT, W, NT, JG>(x, key, c, g), ...);
}

// the register rows rotated left by G columns
template <int RPT, int W, int G>
__device__ __forceinline__ void rotate_rows(float2 (&x)[RPT][W]) {
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
        float2 t[G];
#pragma unroll
        for (int r = 0; r < G; ++r) t[r] = x[s][r];
#pragma unroll
        for (int q = 0; q + G < W; ++q) x[s][q] = x[s][q + G];
#pragma unroll
        for (int r = 0; r < G; ++r) x[s][W - G + r] = t[r];
    }
}

// Panel factorisation for complex64 with the panel's rows in registers
// (m = n - k0 <= RPT x NT): thread t holds the rows at positions t, t + NT
// (relative to k0) of a sub-panel of W columns (RPT x W <= 32 values; one
// sub-panel of 32 for m <= 512 with NT = 128, 256 or 512 threads as m needs,
// two of 16 for m <= 1024).  Per column: a warp-wide max (redux.sync) of
// packed pivot keys (pivot_key) and one barrier give every thread the pivot
// position; its owner publishes the pivot row and 1 / pivot (second barrier);
// the owners of the diagonal and pivot positions exchange their rows whole in
// registers, and every thread scales and updates its own rows with the pivot
// row read from shared memory (a broadcast).  The columns are processed in
// compiled groups of four with the register rows rotated after each group, so
// that every register index is a constant and the code stays small.  Row
// interchanges reach the columns outside the sub-panel without global-memory
// swaps: the columns not yet loaded are gathered through a position ->
// initial-row map, and the first sub-panel (two sub-panels) is held in shared
// memory, where the second one's interchanges are applied, until the panel is
// written back in LAPACK getrf's row order.  The pivot is the largest |v|^2
// to 13 mantissa bits (ties: smallest position), within 2^-13 of the exact
// partial-pivoting choice.
template <int RPT, int W, int NT>
__global__ void __launch_bounds__(NT) panel_reg_kernel(int n, int k0, int kb, float2* A, int* piv, int* info) {
    static_assert(RPT * W <= 32 && (RPT == 1 || W * RPT == kNB), "register panel: RPT x W values per thread");
    static_assert(RPT * NT <= 1024, "pivot keys hold positions below 1024");
    constexpr int NW = NT / 32;
    extern __shared__ unsigned char smraw[];
    const int m = n - k0;
    float2* S1 = reinterpret_cast<float2*>(smraw);   // [W][m]: the first sub-panel (RPT > 1)
    int* perm = reinterpret_cast<int*>(smraw + (RPT > 1 ? sizeof(float2) * (size_t)W * m : 0));
    __shared__ float2 crow[2][W];                    // the pivot row
    __shared__ unsigned ckey[2][NW];                  // each warp's candidate key (pivot_key)
    __shared__ float2 civ[2];                        // 1 / pivot
    __shared__ float2 rowj[2][W];                    // the row at the diagonal position
    __shared__ float2 top[W][W];                     // top rows of the second sub-panel (its U block)
    float2* a = A + (size_t)blockIdx.x * n * n;
    int* pv = piv + (size_t)blockIdx.x * n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 x[RPT][W];
    for (int i = tid; i < m; i += NT) perm[i] = i;
    __syncthreads();
    const int nsub = (kb + W - 1) / W;
    for (int sp = 0; sp < nsub; ++sp) {
        const int s0 = sp * W, ws = min(W, kb - s0);
        // the sub-panel's columns keep the panel's initial row order in global memory
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
            const int i = s * NT + tid;
            const float2* src = a + (size_t)(k0 + s0) * n + k0 + (i < m ? perm[i] : 0);
#pragma unroll
            for (int c = 0; c < W; ++c) x[s][c] = (i < m && c < ws) ? src[(size_t)c * n] : make_float2(0.f, 0.f);
        }
        if constexpr (RPT > 1) {
            if (sp > 0) {
                // top rows (positions < s0, thread = position): U = L11^{-1} A12 with the
                // unit-lower L11 of the first sub-panel, one warp per column, lane = row
                if (tid < s0)
#pragma unroll
                    for (int c = 0; c < W; ++c) top[tid][c] = x[0][c];
                __syncthreads();
                if (warp < ws) {
                    float2 v = lane < s0 ? top[lane][warp] : make_float2(0.f, 0.f);
                    for (int t = 0; t < s0 - 1; ++t) {
                        const float2 vt = make_float2(__shfl_sync(0xffffffffu, v.x, t), __shfl_sync(0xffffffffu, v.y, t));
                        if (lane > t && lane < s0) v = fms(v, S1[(size_t)t * m + lane], vt);
                    }
                    if (lane < s0) top[lane][warp] = v;
                }
                __syncthreads();
                if (tid < s0)
#pragma unroll
                    for (int c = 0; c < W; ++c) x[0][c] = top[tid][c];
                // rows below: x[i][c] -= sum_t L[i][t] U[t][c]
                for (int t = 0; t < s0; ++t) {
#pragma unroll
                    for (int s = 0; s < RPT; ++s) {
                        const int i = s * NT + tid;
                        if (i >= s0 && i < m) {
                            const float2 l = S1[(size_t)t * m + i];
#pragma unroll
                            for (int c = 0; c < W; ++c) x[s][c] = fms(x[s][c], l, top[t][c]);
                        }
                    }
                }
            }
        }
        // this thread's best candidate for the sub-panel's first column
        unsigned key = 0u;
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
            const int i = s * NT + tid;
            if (i >= s0 && i < m) key = max(key, pivot_key(x[s][0], i));
        }
        {
            // columns in groups of kG: one compiled group, the rows rotated by kG
            // after each (W / kG rotations restore the column order)
            constexpr int kG = 4;
            static_assert(W % kG == 0, "whole groups");
            const PanelCtx<RPT, W, NT> c{S1, perm, pv, info, crow, ckey, civ, rowj, m, k0, s0, ws, sp, tid, lane, warp};
#pragma unroll 1
            for (int g = 0; g < W; g += kG) {
                panel_group<RPT, W, NT>(x, key, c, g, std::make_integer_sequence<int, kG>{});
                rotate_rows<RPT, W, kG>(x);
            }
        }
        if constexpr (RPT > 1) {
            if (sp == 0 && nsub > 1) {
#pragma unroll
                for (int s = 0; s < RPT; ++s) {
                    const int i = s * NT + tid;
                    if (i < m)
#pragma unroll
                        for (int c = 0; c < W; ++c) S1[(size_t)c * m + i] = x[s][c];
                }
                __syncthreads();   // S1 and the position map complete before the next sub-panel
                continue;
            }
        }
        // write back (final positions): this sub-panel, then the first one
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
            const int i = s * NT + tid;
            if (i < m) {
                float2* dst = a + (size_t)(k0 + s0) * n + k0 + i;
#pragma unroll
                for (int c = 0; c < W; ++c)
                    if (c < ws) dst[(size_t)c * n] = x[s][c];
            }
        }
        if constexpr (RPT > 1) {
            if (sp > 0) {
                __syncthreads();   // the last interchanges of S1 rows are done
                for (int c = 0; c < W; ++c)
                    for (int i = tid; i < m; i += NT) a[(size_t)(k0 + c) * n + k0 + i] = S1[(size_t)c * m + i];
            }
        }
    }
}

// Sub-panel width of the panel kernel: the widest power of two (at most the
// panel width) whose m x w block fits in about 200 KB of shared memory.
template <typename T>
int panel_width(int m) {
    int w = kNB;
    while (w > 1 && (size_t)m * w * sizeof(T) > 200 * 1024) w >>= 1;
    return w;
}

// Row swaps of the panel applied to the columns outside it, then the
// unit-lower solve U12 = L11^{-1} A12 for the columns right of the panel.
// One CTA of 256 threads per (64-column tile, matrix).  Warp 0 gives every
// row the swaps touch a slot (the kb panel rows, then each distinct pivot row
// below the panel) and replays the swaps on slot indices once, which yields
// the source slot of every destination slot; the tile's slot rows are then
// loaded already permuted, solved and written back.  The solve takes four
// lanes per column (eight rows each, in registers) and broadcasts x_j by
// shuffles inside the group, so it needs no block barrier per step.  The
// tiles start at column col0: 0 applies the interchanges to every column
// outside the panel (LAPACK getrf's row order of L); col0 = k0 + kb to the
// columns right of the panel only, and then the CTAs of tile 0 write the step's
// slot mapping to ptab ([mode][step][2 kNB] pairs (row, row its content comes
// from), (-1, -1) beyond the slots), with which the forward solve applies the
// step's interchanges to the right-hand sides when it reaches the step's block.
constexpr int kSwapCols = 64;

template <typename T>
__global__ void __launch_bounds__(256) swap_trsm_kernel(int n, int k0, int kb, int col0, T* A, const int* piv,
                                                        int2* ptab, unsigned char* bimg, int nblk) {
    extern __shared__ unsigned char smraw[];
    T* blk = reinterpret_cast<T*>(smraw);                 // [kSwapCols][2*kNB]: slots of each column
    T* L = blk + (size_t)kSwapCols * 2 * kNB;             // [kNB][kNB] (col-major), right tiles only
    __shared__ int srow[2 * kNB];                         // global row of each slot
    __shared__ int ssrc[2 * kNB];                         // slot whose content ends in slot r
    __shared__ int sslot[kNB];                            // slot of pivot p_j
    __shared__ int nslots;
    const int b = blockIdx.y;
    T* a = A + (size_t)b * n * n;
    const int* pv = piv + (size_t)b * n;
    const int c0 = col0 + blockIdx.x * kSwapCols;
    const int ncol = min(kSwapCols, n - c0);   // <= 0: a CTA that only writes ptab
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        const int p = lane < kb ? pv[k0 + lane] : -1;
        const bool outside = lane < kb && p >= k0 + kb;
        // lanes holding the same outside pivot row share one slot, numbered in
        // order of first occurrence after the kb panel rows
        const unsigned same = __match_any_sync(0xffffffffu, outside ? p : -1 - lane);
        const int leader = __ffs(same) - 1;
        const unsigned firsts = __ballot_sync(0xffffffffu, outside && leader == lane);
        const int oslot = kb + __popc(firsts & ((1u << leader) - 1u));
        if (lane < kb) {
            srow[lane] = k0 + lane;
            sslot[lane] = outside ? oslot : p - k0;
            if (outside && leader == lane) srow[oslot] = p;
        }
        const int ns = kb + __popc(firsts);
        for (int r = lane; r < ns; r += 32) ssrc[r] = r;
        __syncwarp();
        if (lane == 0) {
            nslots = ns;
            for (int j = 0; j < kb; ++j) {
                const int s2 = sslot[j];
                if (s2 != j) {
                    const int t = ssrc[j];
                    ssrc[j] = ssrc[s2];
                    ssrc[s2] = t;
                }
            }
        }
    }
    __syncthreads();
    const int ns = nslots;
    if (ptab && blockIdx.x == 0 && tid < 2 * kNB) {
        const int steps = (n + kNB - 1) / kNB;
        ptab[((size_t)b * steps + k0 / kNB) * 2 * kNB + tid] =
            tid < ns ? make_int2(srow[tid], srow[ssrc[tid]]) : make_int2(-1, -1);
    }
    const bool right = c0 + ncol > k0 + kb;
    // load the slot rows permuted: slot r of column c at blk[c * 2kNB + r]
    for (int idx = tid; idx < ncol * ns; idx += blockDim.x) {
        const int c = idx / ns, r = idx - c * ns;
        const int col = c0 + c;
        if (col < k0 || col >= k0 + kb) blk[c * 2 * kNB + r] = a[(size_t)col * n + srow[ssrc[r]]];
    }
    if (right)
        for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
            const int j = idx / kb, i = idx - j * kb;      // L[i][j] at L[j*kNB + i]
            L[j * kNB + i] = a[(size_t)(k0 + j) * n + k0 + i];
        }
    __syncthreads();
    if (right) {
        // unit-lower solve on the right columns: lane q of a 4-lane group owns rows q, q+4, ..
        const int c = tid >> 2, q = tid & 3;
        const int col = c0 + c;
        const bool act = c < ncol && col >= k0 + kb;
        T* x = blk + c * 2 * kNB;
        T v[kNB / 4];
#pragma unroll
        for (int t = 0; t < kNB / 4; ++t) {
            const int i = q + 4 * t;
            v[t] = act && i < kb ? x[i] : Cx<T>::mk(0, 0);
        }
        const int base = lane & ~3;
#pragma unroll
        for (int j = 0; j < kNB - 1; ++j) {
            const T own = v[j >> 2];
            const T xj = Cx<T>::mk(__shfl_sync(0xffffffffu, own.x, base | (j & 3)),
                                   __shfl_sync(0xffffffffu, own.y, base | (j & 3)));
#pragma unroll
            for (int t = 0; t < kNB / 4; ++t) {
                const int i = q + 4 * t;
                if (i > j && i < kb) v[t] = fms(v[t], L[j * kNB + i], xj);
            }
        }
        if (act)
#pragma unroll
            for (int t = 0; t < kNB / 4; ++t) {
                const int i = q + 4 * t;
                if (i < kb) x[i] = v[t];
            }
    }
    __syncthreads();
    // write back every slot
    for (int idx = tid; idx < ncol * ns; idx += blockDim.x) {
        const int c = idx / ns, r = idx - c * ns;
        const int col = c0 + c;
        if (col < k0 || col >= k0 + kb) a[(size_t)col * n + srow[r]] = blk[c * 2 * kNB + r];
    }
    if constexpr (sizeof(T) == 8) {
        // complex64 with col0 = k0 + kb: this tile is column block blockIdx.x of the
        // trailing update; its B' image (the TF32 hi / lo split of [Re U12; Im U12]
        // in the update's shared-memory layout, tc_update.cuh) from the solved rows
        if (bimg && ncol > 0) {
            uint4* hi = reinterpret_cast<uint4*>(bimg + ((size_t)b * nblk + blockIdx.x) * tcu::kBImg);
            uint4* lo = hi + tcu::kBBytes / 16;
            for (int u = tid; u < (int)(tcu::kBBytes / 16); u += blockDim.x) {
                const int kc = u >> 6, j = u & 63, kk = (kc * 4) & 31;
                uint32_t h[4], l[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = kk + e;
                    const T v = (j < ncol && k < kb) ? blk[j * 2 * kNB + k] : Cx<T>::mk(0, 0);
                    tcu::split_tf32(kc < 8 ? v.x : v.y, h[e], l[e]);
                }
                hi[u] = make_uint4(h[0], h[1], h[2], h[3]);
                lo[u] = make_uint4(l[0], l[1], l[2], l[3]);
            }
        }
    }
}

// Trailing update A22 -= L21 U12 (K = kb <= 32).  Output tile TILE x TILE per
// CTA of 256 threads (16 x 16), TILE/16 x TILE/16 outputs per thread, operands
// staged in static shared memory (< 48 KB): TILE = 64 for complex64, 32 for
// complex128.
template <typename T> struct GemmTile { static constexpr int v = sizeof(T) == 8 ? 64 : 32; };

template <typename T>
__global__ void gemm_update_kernel(int n, int k0, int kb, T* A) {
    constexpr int TL = GemmTile<T>::v, RPT = TL / 16;
    __shared__ T sL[kNB][TL + 1];
    __shared__ T sU[kNB][TL + 1];
    const int b = blockIdx.z;
    T* a = A + (size_t)b * n * n;
    const int r0 = k0 + kb + blockIdx.x * TL, c0 = k0 + kb + blockIdx.y * TL;
    if (r0 >= n || c0 >= n) return;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < kb * TL; idx += blockDim.x) {
        int kk = idx / TL, i = idx % TL;
        int r = r0 + i;
        sL[kk][i] = r < n ? a[(size_t)(k0 + kk) * n + r] : Cx<T>::mk(0, 0);
    }
    for (int idx = tid; idx < kb * TL; idx += blockDim.x) {
        int j = idx / kb, kk = idx % kb;
        int c = c0 + j;
        sU[kk][j] = c < n ? a[(size_t)c * n + k0 + kk] : Cx<T>::mk(0, 0);
    }
    __syncthreads();
    const int tr = tid % 16, tc = tid / 16;
    T acc[RPT][RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int j = 0; j < RPT; ++j) acc[i][j] = Cx<T>::mk(0, 0);
    for (int kk = 0; kk < kb; ++kk) {
        T l[RPT], u[RPT];
#pragma unroll
        for (int i = 0; i < RPT; ++i) l[i] = sL[kk][tr + 16 * i];
#pragma unroll
        for (int j = 0; j < RPT; ++j) u[j] = sU[kk][tc + 16 * j];
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                acc[i][j].x += l[i].x * u[j].x - l[i].y * u[j].y;
                acc[i][j].y += l[i].x * u[j].y + l[i].y * u[j].x;
            }
    }
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        int c = c0 + tc + 16 * j;
        if (c >= n) continue;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            int r = r0 + tr + 16 * i;
            if (r >= n) continue;
            T* e = a + (size_t)c * n + r;
            *e = sub(*e, acc[i][j]);
        }
    }
}

// Solve LU x = b for every matrix and rhs: the row permutation (gathered
// while loading), then blocked unit-lower forward and upper backward
// substitution.  One CTA (512 threads) per (matrix, group of up to kSolveR
// right-hand sides); B is [b][n][nrhs].  The group's right-hand sides live in
// shared memory ([row][R]) for the whole solve, so each factor element read
// from memory serves all of them; each 32-row diagonal block is solved by one
// warp per right-hand side, then the rows outside it are updated.  When n is
// a multiple of 32 (and, with several right-hand sides, the arithmetic is
// complex64) the update takes two adjacent rows per thread and issues a
// block's column loads in chunks (256 bytes per thread with one right-hand
// side; 16-byte loads for complex64 factors), so that enough bytes are in
// flight to stream the factors at HBM speed; each factor pair then serves
// every right-hand side of the group, and the next diagonal block is fetched
// into registers during the update.  With `dinv` (the inverses of the 32 x 32
// diagonal blocks of L and U, diag_inv_kernel; n a multiple of 32) a
// diagonal block is applied as a matrix-vector product by one warp per
// right-hand side, 32 independent products instead of a 32-step dependent
// substitution that the other warps wait for.  Matrices whose active flag is
// 0 are skipped (converged modes).
constexpr int kSolveR = 8;

template <typename T> __device__ __forceinline__ T widen(float2 v) { return Cx<T>::mk(v.x, v.y); }
template <typename T> __device__ __forceinline__ T widen(double2 v) { return Cx<T>::mk(v.x, v.y); }

// two adjacent column entries p[0], p[1] (p 16-byte aligned for complex64)
__device__ __forceinline__ void load_pair(const float2* p, float2& u, float2& v) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    u = make_float2(q.x, q.y);
    v = make_float2(q.z, q.w);
}
__device__ __forceinline__ void load_pair(const double2* p, double2& u, double2& v) {
    u = __ldg(p);
    v = __ldg(p + 1);
}

// x[i][q], x[i+1][q] -= sum_{c < kNB} F[c][i..i+1] xs[c][q] for the group's
// right-hand sides q < nr (a full 32-column block; xs row stride R), factor
// loads issued in chunks of 256 bytes per thread
template <typename T, typename TF, int RM>
__device__ __forceinline__ void block_pair_update(const TF* col, int n, const T* xs, int R, int nr, T (&acc0)[RM],
                                                  T (&acc1)[RM]) {
    constexpr int CH = RM == 1 ? (int)(256 / (2 * sizeof(TF))) : 2;
#pragma unroll
    for (int c0 = 0; c0 < kNB; c0 += CH) {
        TF l0[CH], l1[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) load_pair(col + (size_t)(c0 + c) * n, l0[c], l1[c]);
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const T f0 = widen<T>(l0[c]), f1 = widen<T>(l1[c]);
#pragma unroll
            for (int q = 0; q < RM; ++q)
                if (q < nr) {
                    const T xc = xs[(c0 + c) * R + q];
                    acc0[q] = fms(acc0[q], f0, xc);
                    acc1[q] = fms(acc1[q], f1, xc);
                }
        }
    }
}

template <typename T, typename TF, int RM>
__global__ void __launch_bounds__(512) lu_solve_kernel(int n, int nrhs, int Rg, const TF* LU, const int* perm,
                                                       T* B, const int* active, const TF* dinv, const int2* ptab) {
    const int R = RM == 1 ? 1 : Rg;    // compile-time 1 in the single-wave variant
    const int b = blockIdx.x, r0 = blockIdx.y * R, nr = RM == 1 ? 1 : min(R, nrhs - r0);
    if (active && !active[b]) return;
    extern __shared__ unsigned char smraw[];
    T* sx = reinterpret_cast<T*>(smraw);                     // n x R entries, sx[i * R + q]
    const TF* a = LU + (size_t)b * n * n;
    const int* pm = perm + (size_t)b * n;
    T* x = B + (size_t)b * n * nrhs;
    __shared__ __align__(16) TF sD[kNB * kNB];     // diagonal block, sD[col * kNB + row]
    constexpr int kDiagPer = (int)(kNB * kNB * sizeof(TF) / (512 * 16));   // 16-byte pieces per thread
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nblk = (n + kNB - 1) / kNB;
    // with ptab the factor's L columns keep the row order of their step: the
    // right-hand sides are loaded as they are and each step's interchanges are
    // applied when the forward solve reaches its block; else loaded permuted
    const int2* pt = ptab ? ptab + (size_t)b * nblk * 2 * kNB : nullptr;
    for (int idx = tid; idx < n * nr; idx += blockDim.x) {
        const int i = idx / nr, q = idx - i * nr;
        sx[i * R + q] = x[(size_t)(pt ? i : pm[i]) * nrhs + r0 + q];
    }
    // the pair path: full blocks only, and with several right-hand sides only
    // for complex64 accumulators (register budget of 512 threads)
    const bool vec = (n % kNB) == 0 && (RM == 1 || sizeof(T) == 8);
    // (complex64 factors only: the FP64 path keeps the substitution)
    const bool inv = std::is_same<TF, float2>::value && vec && dinv != nullptr;
    // diagonal block j0 into registers (16-byte pieces, column by column): the
    // factor's block, or with inv the inverse of its L (t = 0) or U (t = 1) part
    const TF* dinv_b = inv ? dinv + (size_t)b * nblk * 2 * kNB * kNB : nullptr;
    auto fetch_diag = [&](int j0, int jb, int t, float4 (&reg)[kDiagPer]) {
        if (inv) {
            // the inverse blocks are contiguous: full 16-byte pieces
            const float4* src = reinterpret_cast<const float4*>(dinv_b + ((size_t)(j0 / kNB) * 2 + t) * kNB * kNB);
#pragma unroll
            for (int q = 0; q < kDiagPer; ++q) reg[q] = __ldg(src + tid + q * 512);
            return;
        }
#pragma unroll
        for (int q = 0; q < kDiagPer; ++q) {
            const int e = (tid + q * 512) * (int)(16 / sizeof(TF));     // first element of the piece
            const int c = e / kNB, i = e - c * kNB;
            reg[q] = (c < jb && i < jb) ? __ldg(reinterpret_cast<const float4*>(a + (size_t)(j0 + c) * n + j0 + i))
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    // x_blk <- Inv x_blk for the warp's right-hand side (inv path)
    auto apply_inv = [&](int j0) {
        if (warp < nr) {
            const T v = sx[(j0 + lane) * R + warp];
            T acc0 = Cx<T>::mk(0, 0), acc1 = acc0;
#pragma unroll
            for (int c = 0; c < kNB; c += 2) {
                const T x0 = Cx<T>::mk(__shfl_sync(0xffffffff, v.x, c), __shfl_sync(0xffffffff, v.y, c));
                const T x1 = Cx<T>::mk(__shfl_sync(0xffffffff, v.x, c + 1), __shfl_sync(0xffffffff, v.y, c + 1));
                acc0 = fma_c(acc0, widen<T>(sD[c * kNB + lane]), x0);
                acc1 = fma_c(acc1, widen<T>(sD[(c + 1) * kNB + lane]), x1);
            }
            sx[(j0 + lane) * R + warp] = add(acc0, acc1);
        }
    };
    auto store_diag = [&](const float4 (&reg)[kDiagPer]) {
#pragma unroll
        for (int t = 0; t < kDiagPer; ++t) reinterpret_cast<float4*>(sD)[tid + t * 512] = reg[t];
    };
    float4 dreg[kDiagPer];
    int2 pn0 = make_int2(-1, -1), pn1 = pn0;   // interchange entries of the next block (ptab)
    if (pt && warp < nr) {
        pn0 = pt[lane];
        pn1 = pt[32 + lane];
    }
    // forward: L y = x (unit diagonal)
    if (vec) {
        fetch_diag(0, kNB, 0, dreg);
        store_diag(dreg);
    }
    __syncthreads();
    for (int j0 = 0; j0 < n; j0 += kNB) {
        const int jb = min(kNB, n - j0);
        if (!vec) {
            for (int idx = tid; idx < jb * jb; idx += blockDim.x) {
                const int c = idx / jb, i = idx % jb;
                sD[c * kNB + i] = a[(size_t)(j0 + c) * n + j0 + i];
            }
            __syncthreads();
        }
        if (pt && warp < nr) {
            // this step's interchanges on the warp's right-hand side: slots lane, lane + 32
            // (entries loaded one block ahead, off the critical path)
            const int2 e0 = pn0, e1 = pn1;
            if (j0 + kNB < n) {
                pn0 = pt[(size_t)(j0 / kNB + 1) * 2 * kNB + lane];
                pn1 = pt[(size_t)(j0 / kNB + 1) * 2 * kNB + 32 + lane];
            }
            const T v0 = e0.x >= 0 ? sx[e0.y * R + warp] : Cx<T>::mk(0, 0);
            const T v1 = e1.x >= 0 ? sx[e1.y * R + warp] : Cx<T>::mk(0, 0);
            __syncwarp();
            if (e0.x >= 0) sx[e0.x * R + warp] = v0;
            if (e1.x >= 0) sx[e1.x * R + warp] = v1;
            __syncwarp();
        }
        if (inv) {
            apply_inv(j0);
        } else if (warp < nr) {
            T v = lane < jb ? sx[(j0 + lane) * R + warp] : Cx<T>::mk(0, 0);
            for (int c = 0; c < jb; ++c) {
                T xc = Cx<T>::mk(__shfl_sync(0xffffffff, v.x, c), __shfl_sync(0xffffffff, v.y, c));
                if (lane > c && lane < jb) v = fms(v, widen<T>(sD[c * kNB + lane]), xc);
            }
            if (lane < jb) sx[(j0 + lane) * R + warp] = v;
        }
        __syncthreads();
        if (vec) {
            const bool more = j0 + kNB < n;
            if (more) fetch_diag(j0 + kNB, kNB, 0, dreg);
            for (int i = j0 + kNB + 2 * tid; i < n; i += 2 * blockDim.x) {
                T acc0[RM], acc1[RM];
#pragma unroll
                for (int q = 0; q < RM; ++q)
                    if (q < nr) acc0[q] = sx[i * R + q], acc1[q] = sx[(i + 1) * R + q];
                block_pair_update<T, TF, RM>(a + (size_t)j0 * n + i, n, sx + (size_t)j0 * R, R, nr, acc0, acc1);
#pragma unroll
                for (int q = 0; q < RM; ++q)
                    if (q < nr) sx[i * R + q] = acc0[q], sx[(i + 1) * R + q] = acc1[q];
            }
            __syncthreads();
            if (more) store_diag(dreg);
        } else {
            for (int i = j0 + jb + tid; i < n; i += blockDim.x) {
                T acc[RM];
#pragma unroll
                for (int q = 0; q < RM; ++q)
                    if (q < nr) acc[q] = sx[i * R + q];
#pragma unroll 8
                for (int c = 0; c < jb; ++c) {
                    const T l = widen<T>(a[(size_t)(j0 + c) * n + i]);
#pragma unroll
                    for (int q = 0; q < RM; ++q)
                        if (q < nr) acc[q] = fms(acc[q], l, sx[(j0 + c) * R + q]);
                }
#pragma unroll
                for (int q = 0; q < RM; ++q)
                    if (q < nr) sx[i * R + q] = acc[q];
            }
        }
        __syncthreads();
    }
    // backward: U x = y
    if (vec) {
        fetch_diag((nblk - 1) * kNB, kNB, 1, dreg);
        store_diag(dreg);
        __syncthreads();
    }
    for (int bi = nblk - 1; bi >= 0; --bi) {
        const int j0 = bi * kNB, jb = min(kNB, n - j0);
        if (!vec) {
            for (int idx = tid; idx < jb * jb; idx += blockDim.x) {
                const int c = idx / jb, i = idx % jb;
                sD[c * kNB + i] = a[(size_t)(j0 + c) * n + j0 + i];
            }
            __syncthreads();
        }
        if (inv) {
            apply_inv(j0);
        } else if (warp < nr) {
            T v = lane < jb ? sx[(j0 + lane) * R + warp] : Cx<T>::mk(0, 0);
            for (int c = jb - 1; c >= 0; --c) {
                if (lane == c) v = mul(v, rcp(widen<T>(sD[c * kNB + c])));
                T xc = Cx<T>::mk(__shfl_sync(0xffffffff, v.x, c), __shfl_sync(0xffffffff, v.y, c));
                if (lane < c) v = fms(v, widen<T>(sD[c * kNB + lane]), xc);
            }
            if (lane < jb) sx[(j0 + lane) * R + warp] = v;
        }
        __syncthreads();
        if (vec) {
            if (bi > 0) fetch_diag(j0 - kNB, kNB, 1, dreg);
            for (int i = 2 * tid; i < j0; i += 2 * blockDim.x) {
                T acc0[RM], acc1[RM];
#pragma unroll
                for (int q = 0; q < RM; ++q)
                    if (q < nr) acc0[q] = sx[i * R + q], acc1[q] = sx[(i + 1) * R + q];
                block_pair_update<T, TF, RM>(a + (size_t)j0 * n + i, n, sx + (size_t)j0 * R, R, nr, acc0, acc1);
#pragma unroll
                for (int q = 0; q < RM; ++q)
                    if (q < nr) sx[i * R + q] = acc0[q], sx[(i + 1) * R + q] = acc1[q];
            }
            __syncthreads();
            if (bi > 0) store_diag(dreg);
        } else {
            for (int i = tid; i < j0; i += blockDim.x) {
                T acc[RM];
#pragma unroll
                for (int q = 0; q < RM; ++q)
                    if (q < nr) acc[q] = sx[i * R + q];
#pragma unroll 8
                for (int c = 0; c < jb; ++c) {
                    const T u = widen<T>(a[(size_t)(j0 + c) * n + i]);
#pragma unroll
                    for (int q = 0; q < RM; ++q)
                        if (q < nr) acc[q] = fms(acc[q], u, sx[(j0 + c) * R + q]);
                }
#pragma unroll
                for (int q = 0; q < RM; ++q)
                    if (q < nr) sx[i * R + q] = acc[q];
            }
        }
        __syncthreads();
    }
    for (int idx = tid; idx < n * nr; idx += blockDim.x) {
        const int i = idx / nr, q = idx - i * nr;
        x[(size_t)i * nrhs + r0 + q] = sx[i * R + q];
    }
}

// Inverses of the kNB x kNB diagonal blocks of every complex64 factor (n a
// multiple of kNB), for the solves' matrix-vector diagonal steps: grid
// (n / kNB, batch), two warps; warp 0 inverts the unit lower part L_kk, warp 1
// the upper part U_kk.  Lane j forms column j of the inverse by substitution
// on e_j held in registers (all lanes take the same steps and read the block
// as shared-memory broadcasts).  Output [b][k][2][col][row], column-major per
// block like the factor.  A zero pivot gives non-finite entries, as the
// substitution would.
__global__ void __launch_bounds__(64) diag_inv_kernel(int n, const float2* LU, float2* dinv) {
    __shared__ float2 sB[kNB * kNB];    // [col * kNB + row]
    const int k = blockIdx.x, b = blockIdx.y, nblk = n / kNB;
    const float2* a = LU + (size_t)b * n * n + (size_t)k * kNB * n + (size_t)k * kNB;
    for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
        const int c = idx / kNB, r = idx - c * kNB;
        sB[idx] = a[(size_t)c * n + r];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, j = threadIdx.x & 31;
    float2 y[kNB];
#pragma unroll
    for (int r = 0; r < kNB; ++r) y[r] = make_float2(r == j ? 1.0f : 0.0f, 0.0f);
    if (warp == 0) {
        // L y = e_j (unit diagonal): y_r -= L[r][c] y_c for r > c, c ascending
#pragma unroll
        for (int c = 0; c < kNB; ++c)
#pragma unroll
            for (int r = c + 1; r < kNB; ++r) y[r] = fms(y[r], sB[c * kNB + r], y[c]);
    } else {
        // U y = e_j: y_c /= U[c][c], then y_r -= U[r][c] y_c for r < c, c descending
#pragma unroll
        for (int c = kNB - 1; c >= 0; --c) {
            y[c] = mul(y[c], rcp(sB[c * kNB + c]));
#pragma unroll
            for (int r = 0; r < c; ++r) y[r] = fms(y[r], sB[c * kNB + r], y[c]);
        }
    }
    float2* o = dinv + (((size_t)b * nblk + k) * 2 + warp) * kNB * kNB + (size_t)j * kNB;
#pragma unroll
    for (int r = 0; r < kNB; ++r) o[r] = y[r];
}

__global__ void c128_to_c64_kernel(int64_t count, const double2* s, float2* d) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < count; i += stride) d[i] = make_float2((float)s[i].x, (float)s[i].y);
}

// R -= A X over one chunk of kResCols columns (R starts as B): grid (row
// blocks, column chunks, matrices), so a single active matrix still spreads
// over many SMs (the GB300's FP64 pipe is 2 FMA/clk per SM).
constexpr int kResCols = 32;
__global__ void residual_kernel(int n, int nrhs, const double2* A, const double2* X, double2* R, const int* active) {
    const int b = blockIdx.z;
    if (active && !active[b]) return;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * nrhs) return;
    const int r = (int)(idx % nrhs), row = (int)(idx / nrhs);
    const int c0 = blockIdx.y * kResCols, c1 = min(n, c0 + kResCols);
    const double2* a = A + (size_t)b * n * n;
    const double2* x = X + (size_t)b * n * nrhs;
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll 16
    for (int c = c0; c < c1; ++c) acc = fms(acc, __ldg(a + (size_t)c * n + row), x[(size_t)c * nrhs + r]);
    double* o = reinterpret_cast<double*>(R + (size_t)b * n * nrhs + idx);
    atomicAdd(o, acc.x);
    atomicAdd(o + 1, acc.y);
}

// |R|^2, |B|^2, |X|^2 per (matrix, rhs): grid (batch, nrhs), 256 threads
__global__ void norms3_kernel(int n, int nrhs, const double2* R, const double2* B, const double2* X, double* rn2,
                              double* bn2, double* xn2, const int* active) {
    __shared__ double sh[3][8];
    const int b = blockIdx.x, r = blockIdx.y;
    if (active && !active[b]) return;
    const size_t base = (size_t)b * n * nrhs + r;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int row = threadIdx.x; row < n; row += blockDim.x) {
        const size_t i = base + (size_t)row * nrhs;
        s0 += R[i].x * R[i].x + R[i].y * R[i].y;
        s1 += B[i].x * B[i].x + B[i].y * B[i].y;
        s2 += X[i].x * X[i].x + X[i].y * X[i].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffff, s0, o);
        s1 += __shfl_xor_sync(0xffffffff, s1, o);
        s2 += __shfl_xor_sync(0xffffffff, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s0;
        sh[1][threadIdx.x >> 5] = s1;
        sh[2][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t0 += sh[0][w], t1 += sh[1][w], t2 += sh[2][w];
        const size_t k = (size_t)b * nrhs + r;
        rn2[k] = t0;
        bn2[k] = t1;
        xn2[k] = t2;
    }
}

// float nearest to the double whose 32-bit halves are (lo, hi), with 32-bit
// integer operations only (on this GPU a double -> float conversion issues to
// the FP64 pipe): round to nearest even on the 29 dropped significand bits;
// results below float's normal range flush to a signed zero, above it give
// infinity; NaN stays NaN.
__device__ __forceinline__ float f32_of_halves(uint32_t lo, uint32_t hi) {
    const uint32_t sg = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    if (e == 0x7ff) return __uint_as_float(sg | (((hi & 0xfffffu) | lo) ? 0x7fc00000u : 0x7f800000u));
    const int ef = e - 1023 + 127;
    if (ef >= 255) return __uint_as_float(sg | 0x7f800000u);
    if (ef <= 0) return __uint_as_float(sg);
    const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29), rest = lo & 0x1fffffffu;
    uint32_t bits = ((uint32_t)ef << 23) | m;
    if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) bits += 1u;   // a carry moves into the exponent
    return __uint_as_float(sg | bits);
}

// complex64 copy of every matrix and |A_b|_F^2 in the same pass over A:
// grid (blocks per matrix, matrices), out zeroed beforehand.  The entries are
// read as 32-bit words and converted with integer operations; the squares
// accumulate in FP32 per thread (the norm enters only the backward-error test
// of the refinement, where 1e-5 relative is ample) and in FP64 across warps.
__global__ void c64_fro2_kernel(int64_t per, const double2* A, float2* A32, double* out) {
    __shared__ double sh[8];
    const uint4* a = reinterpret_cast<const uint4*>(A + (size_t)blockIdx.y * per);
    float2* d = A32 + (size_t)blockIdx.y * per;
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 v = __ldcs(a + i);      // read once: streaming
        const float2 f = make_float2(f32_of_halves(v.x, v.y), f32_of_halves(v.z, v.w));
        d[i] = f;
        acc = __fmaf_rn(f.x, f.x, __fmaf_rn(f.y, f.y, acc));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffff, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        atomicAdd(out + blockIdx.y, t);
    }
}

__global__ void add_correction_kernel(int64_t count, int64_t per_matrix, const float2* d, double2* X,
                                      const int* active) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count && (!active || active[i / per_matrix])) {
        X[i].x += (double)d[i].x;
        X[i].y += (double)d[i].y;
    }
}

}  // namespace

// Swap sequence -> row permutation, in place: piv[b][j] = row swapped with row
// j at step j becomes perm[b][i] = original row that ends in row i (replayed by
// one thread per matrix on a shared-memory index array).
__global__ void perm_kernel(int n, int* piv) {
    extern __shared__ int sp[];
    int* p = piv + (size_t)blockIdx.x * n;
    int* sw = sp + n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sp[i] = i;
        sw[i] = p[i];
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int j = 0; j < n; ++j) {
            const int q = sw[j];
            const int t = sp[j];
            sp[j] = sp[q];
            sp[q] = t;
        }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = sp[i];
}

// Dynamic shared-memory limits of the factorisation's kernels, set once per
// process (outside any stream capture of the factorisation).
template <typename T>
cudaError_t lu_prepare() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        cudaError_t e;
        if ((e = allow_max_smem(panel_kernel<T>)) == cudaSuccess && (e = allow_max_smem(swap_trsm_kernel<T>)) ==
            cudaSuccess && (e = allow_max_smem(perm_kernel)) == cudaSuccess) {
            if constexpr (sizeof(T) == 8) {
                if ((e = allow_max_smem(tcu::update_kernel)) == cudaSuccess &&
                    (e = allow_max_smem(panel_reg_kernel<1, kNB, 128>)) == cudaSuccess &&
                    (e = allow_max_smem(panel_reg_kernel<1, kNB, 256>)) == cudaSuccess &&
                    (e = allow_max_smem(panel_reg_kernel<1, kNB, kPanelThreads>)) == cudaSuccess)
                    e = allow_max_smem(panel_reg_kernel<2, kNB / 2, kPanelThreads>);
            }
        }
        err = e;
    });
    return err;
}

namespace {

// cuTensorMapEncodeTiled from the driver, looked up once
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// TMA map of the batch of n x n complex64 matrices as a [batch][n][n] tensor
// of 8-byte elements (row index fastest), 64 x 64 boxes; n must be even (row
// stride a multiple of 16 bytes)
cudaError_t trailing_tensor_map(CUtensorMap* tm, float2* A, int n, int batch) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || (n & 1)) return cudaErrorInvalidValue;
    const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {(cuuint64_t)n * 8, (cuuint64_t)n * n * 8};
    const cuuint32_t box[3] = {tcu::kTileC, tcu::kTileC, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, A, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

// An update-timing event: an external event (an event-record node) when s is
// being captured into a graph, a plain record otherwise (the external flag is
// not valid outside a capture)
static cudaError_t record_update_event(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(s, &st);
    if (ce != cudaSuccess) return ce;
    return st == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                               : cudaEventRecord(e, s);
}

size_t lu_ptab_elems(int n, int batch) { return (size_t)batch * ((n + kNB - 1) / kNB) * 2 * kNB; }

size_t lu_image_bytes(int n, int batch) {
    const int nblk = n > kNB ? tcu::update_blocks(n, 0, kNB) : 0;
    return (size_t)batch * nblk * (tcu::kAImg + tcu::kBImg);
}

template <typename T>
cudaError_t batched_lu(int n, int batch, T* A, int* piv, int* info, cudaStream_t s, unsigned char* img,
                       int2* ptab, const LuSide* side, cudaEvent_t* upd_ev) {
    cudaError_t pe = lu_prepare<T>();
    if (pe != cudaSuccess) return pe;
    if constexpr (sizeof(T) == 8) {
        if (!ptab) return cudaErrorInvalidValue;
    } else {
        ptab = nullptr;
    }
    // complex64: the trailing matrix as a TMA tensor, and the SMs for the
    // persistent update
    CUtensorMap tmA;
    int sms = 0;
    if constexpr (sizeof(T) == 8) {
        if (n > kNB) {
            if (!img || (reinterpret_cast<uintptr_t>(img) & 15)) return cudaErrorInvalidValue;
            cudaError_t e = trailing_tensor_map(&tmA, reinterpret_cast<float2*>(A), n, batch);
            int dev = 0;
            if (e == cudaSuccess) e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
        }
    }
    for (int k0 = 0; k0 < n; k0 += kNB) {
        int kb = std::min(kNB, n - k0);
        const int m = n - k0;
        bool reg_panel = false;
        if constexpr (sizeof(T) == 8) {
            // complex64 panels of up to 2 x 512 rows: rows in registers
            float2* A32 = reinterpret_cast<float2*>(A);
            // one row per thread up to 512 rows (128 / 256 / 512 threads), then two
            const size_t smi = sizeof(int) * (size_t)m;
            reg_panel = true;
            if (m <= 128)
                panel_reg_kernel<1, kNB, 128><<<batch, 128, smi, s>>>(n, k0, kb, A32, piv, info);
            else if (m <= 256)
                panel_reg_kernel<1, kNB, 256><<<batch, 256, smi, s>>>(n, k0, kb, A32, piv, info);
            else if (m <= kPanelThreads)
                panel_reg_kernel<1, kNB, kPanelThreads><<<batch, kPanelThreads, smi, s>>>(n, k0, kb, A32, piv, info);
            else if (m <= 2 * kPanelThreads)
                panel_reg_kernel<2, kNB / 2, kPanelThreads>
                    <<<batch, kPanelThreads, smi + sizeof(float2) * (kNB / 2) * (size_t)m, s>>>(n, k0, kb, A32, piv, info);
            else
                reg_panel = false;
        }
        if (!reg_panel) {
            const int w = panel_width<T>(m);
            const size_t smp = sizeof(T) * (size_t)m * w;
            panel_kernel<T><<<batch, kPanelThreads, smp, s>>>(n, k0, kb, w, A, piv, info);
        }
        count_launch(2);
        // complex64: the interchanges reach the right columns only (the solve
        // applies them to the right-hand sides from ptab), and each 64-column tile
        // writes the B' image of its column block of the update; complex128: all columns
        const int col0 = ptab ? k0 + kb : 0;
        const int nblk = n - k0 - kb > 0 ? tcu::update_blocks(n, k0, kb) : 0;
        unsigned char* bimg = ptab && nblk > 0 ? img + (size_t)batch * nblk * tcu::kAImg : nullptr;
        // the A' images need only the panel: with a side stream they run beside
        // the row-swap / block-row-solve kernel
        const bool aside = ptab && nblk > 0 && side && side->stream;
        if (aside) {
            cudaError_t ee;
            if ((ee = cudaEventRecord(side->fork, s)) != cudaSuccess ||
                (ee = cudaStreamWaitEvent(side->stream, side->fork, 0)) != cudaSuccess)
                return ee;
            tcu::operand_image_kernel<<<dim3(nblk, 2, batch), 256, 0, side->stream>>>(
                n, k0, kb, nblk, reinterpret_cast<const float2*>(A), img);
            count_launch();
            if ((ee = cudaEventRecord(side->join, side->stream)) != cudaSuccess) return ee;
        }
        dim3 g1((unsigned)std::max(1, (n - col0 + kSwapCols - 1) / kSwapCols), batch);
        size_t sm1 = sizeof(T) * ((size_t)kSwapCols * 2 * kNB + kNB * kNB);
        swap_trsm_kernel<T><<<g1, 256, sm1, s>>>(n, k0, kb, col0, A, piv, ptab, bimg, nblk);
        int rem = n - k0 - kb;
        if (aside) {
            cudaError_t ee = cudaStreamWaitEvent(s, side->join, 0);
            if (ee != cudaSuccess) return ee;
        }
        if (rem > 0) {
            cudaError_t ee;
            if (upd_ev && (ee = record_update_event(upd_ev[2 * (k0 / kNB)], s)) != cudaSuccess) return ee;
            if constexpr (sizeof(T) == 8) {
                // complex64: the A' images of this step (unless on the side stream;
                // the B' images came with the block-row solve), then the tensor-core
                // update (tcgen05, TF32 split to FP32 accuracy) reading them
                if (!aside) {
                    tcu::operand_image_kernel<<<dim3(nblk, 2, batch), 256, 0, s>>>(
                        n, k0, kb, nblk, reinterpret_cast<const float2*>(A), img);
                    count_launch();
                }
                const long long units = (long long)batch * nblk;
                const int grid = (int)std::min<long long>(units, sms);
                tcu::update_kernel<<<grid, tcu::kPipeThreads, tcu::kPipeSmem, s>>>(tmA, k0, kb, nblk, batch, img,
                                                                                   bimg, info);
            } else {
                constexpr int TL = GemmTile<T>::v;
                dim3 g2((rem + TL - 1) / TL, (rem + TL - 1) / TL, batch);
                gemm_update_kernel<T><<<g2, 256, 0, s>>>(n, k0, kb, A);
            }
            count_launch();
            if (upd_ev && (ee = record_update_event(upd_ev[2 * (k0 / kNB) + 1], s)) != cudaSuccess) return ee;
        }
    }
    if (!ptab) {
        const size_t smq = 2 * sizeof(int) * (size_t)n;
        perm_kernel<<<batch, 256, smq, s>>>(n, piv);
        count_launch();
    }
    return cudaGetLastError();
}

template <typename T, typename TF>
cudaError_t batched_lu_solve(int n, int batch, int nrhs, const TF* LU, const int* piv, T* B,
                             cudaStream_t s, const int* active, const TF* dinv, const int2* ptab) {
    // right-hand sides per CTA: up to kSolveR, as many as fit in shared memory
    // (about 200 KB for the group)
    int R = std::min(nrhs, kSolveR);
    while (R > 1 && sizeof(T) * (size_t)R * (size_t)n > 200 * 1024) --R;
    dim3 g(batch, (nrhs + R - 1) / R);
    // dynamic: right-hand sides; static: the 32 x 32 diagonal block
    size_t sm = sizeof(T) * (size_t)R * (size_t)n;
    const bool big = sm + sizeof(TF) * kNB * kNB > 48 * 1024;
    if (R == 1) {   // the common single-wave case, without the group loops
        if (big) {
            cudaError_t e = allow_max_smem(lu_solve_kernel<T, TF, 1>);
            if (e != cudaSuccess) return e;
        }
        lu_solve_kernel<T, TF, 1><<<g, 512, sm, s>>>(n, nrhs, R, LU, piv, B, active, dinv, ptab);
    } else {
        if (big) {
            cudaError_t e = allow_max_smem(lu_solve_kernel<T, TF, kSolveR>);
            if (e != cudaSuccess) return e;
        }
        lu_solve_kernel<T, TF, kSolveR><<<g, 512, sm, s>>>(n, nrhs, R, LU, piv, B, active, dinv, ptab);
    }
    count_launch();
    return cudaGetLastError();
}

template cudaError_t lu_prepare<double2>();
template cudaError_t lu_prepare<float2>();
template cudaError_t batched_lu<double2>(int, int, double2*, int*, int*, cudaStream_t, unsigned char*, int2*,
                                          const LuSide*, cudaEvent_t*);
template cudaError_t batched_lu<float2>(int, int, float2*, int*, int*, cudaStream_t, unsigned char*, int2*,
                                         const LuSide*, cudaEvent_t*);
template cudaError_t batched_lu_solve<double2, double2>(int, int, int, const double2*, const int*, double2*,
                                                        cudaStream_t, const int*, const double2*, const int2*);
template cudaError_t batched_lu_solve<float2, float2>(int, int, int, const float2*, const int*, float2*,
                                                      cudaStream_t, const int*, const float2*, const int2*);
template cudaError_t batched_lu_solve<double2, float2>(int, int, int, const float2*, const int*, double2*,
                                                       cudaStream_t, const int*, const float2*, const int2*);

cudaError_t convert_to_c64(int64_t count, const double2* src, float2* dst, cudaStream_t s) {
    int blocks = (int)std::min<int64_t>((count + 255) / 256, 152 * 32);
    c128_to_c64_kernel<<<blocks, 256, 0, s>>>(count, src, dst);
    count_launch();
    return cudaGetLastError();
}

cudaError_t residual_c128(int n, int batch, int nrhs, const double2* A, const double2* X,
                          const double2* B, double2* R, double* rnorm, double* bnorm, double* xnorm,
                          cudaStream_t s, const int* active) {
    cudaError_t e = cudaMemcpyAsync(R, B, sizeof(double2) * (size_t)batch * n * nrhs, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    dim3 g((unsigned)(((size_t)n * nrhs + 255) / 256), (unsigned)((n + kResCols - 1) / kResCols), batch);
    residual_kernel<<<g, 256, 0, s>>>(n, nrhs, A, X, R, active);
    norms3_kernel<<<dim3(batch, nrhs), 256, 0, s>>>(n, nrhs, R, B, X, rnorm, bnorm, xnorm, active);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t convert_fro2_c128(int n, int batch, const double2* A, float2* A32, double* out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * batch, s);
    if (e != cudaSuccess) return e;
    const int64_t per = (int64_t)n * n;
    // about 32 CTAs of 256 threads per SM over all matrices (enough loads in flight)
    const int64_t want = std::max<int64_t>(1, (152 * 32 + batch - 1) / batch);
    dim3 g((unsigned)std::min<int64_t>((per + 255) / 256, want), batch);
    c64_fro2_kernel<<<g, 256, 0, s>>>(per, A, A32, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t batched_diag_inv(int n, int batch, const float2* LU, float2* dinv, cudaStream_t s) {
    if (n % kNB != 0) return cudaErrorInvalidValue;
    dim3 g((unsigned)(n / kNB), (unsigned)batch);
    diag_inv_kernel<<<g, 64, 0, s>>>(n, LU, dinv);
    count_launch();
    return cudaGetLastError();
}

cudaError_t refine_step(int n, int batch, int nrhs, const float2* LU32, const int* piv,
                        const double2* R, float2* work32, double2* X, cudaStream_t s, const int* active,
                        const float2* dinv, const int2* ptab) {
    int64_t cnt = (int64_t)batch * n * nrhs;
    cudaError_t e = convert_to_c64(cnt, R, work32, s);
    if (e != cudaSuccess) return e;
    e = batched_lu_solve<float2, float2>(n, batch, nrhs, LU32, piv, work32, s, active, dinv, ptab);
    if (e != cudaSuccess) return e;
    add_correction_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(cnt, (int64_t)n * nrhs, work32, X, active);
    count_launch();
    return cudaGetLastError();
}

}  // namespace pmlbie
