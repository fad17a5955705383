// Float-float kernels of the mixed path (sm_103a): the far-pair modal kernels
// (Green's-function sampling, even-sequence DFTs and the block scatter) in
// the FP32-pair arithmetic of ffloat.cuh, for the GB300 whose FP32 pipe
// retires 64 times the FP64 pipe's operations.  Same mathematics, layout and
// outputs as far_kernel (kernels.cu):
//
//   Sec. 3.1 / 4.3  G~ = e^{i w |dr|}/(4 pi |dr|), |dr|^2 = d~^2 + 4 rho~ rho~' sin^2(psi/2)
//   Sec. 4.1        K~ = N_D(psi) e^{iq}(1 - iq) / (4 pi |dr|^3), modes by the
//                   M-point rule in psi (far pairs)
//
// Scaling.  Each unordered pair is sampled in units of L = 2^eL with
// L^2 ~ |d~^2| + 4 |rho~ rho~'| (so |dr| / L <= ~2 and 1/|dr|^3 stays in float
// range for pairs next to the axis), and e^{-Im q} is carried as a mantissa
// times 2^E per sample; before the transforms every sample of a pair and
// medium is rescaled to the largest E of its sequence (exact powers of two),
// and that exponent, with the powers of L, goes into the exponent field of
// the FP64 results.  The entries leave the kernel as complex128 built from
// the float pairs by integer operations.
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"
#include "device_common.cuh"
#include "ffloat.cuh"

namespace pmlbie {

namespace {

using namespace ffm;

// sin(2 pi / 3) as a float pair
constexpr float kS3Hi = 0x1.bb67aep-1f;
constexpr float kS3Lo = 0x1.0b0996p-26f;

__device__ __forceinline__ cff ldc(const float4* p, int i) { return unpack(p[i]); }
__device__ __forceinline__ void stc(float4* p, int i, cff v) { p[i] = pack(v); }
__device__ __forceinline__ cff czero() { return cff{ff{0.f, 0.f}, ff{0.f, 0.f}}; }
// a - i b and a + i b
__device__ __forceinline__ cff sub_i(cff a, cff b) { return cff{add(a.re, b.im), sub(a.im, b.re)}; }
__device__ __forceinline__ cff add_i(cff a, cff b) { return cff{sub(a.re, b.im), add(a.im, b.re)}; }

// One Stockham stage.  lgNs = log2(Ns) when Ns is a power of two (the radix-4
// and radix-2 stages, which come first), else -1: integer division and
// remainder by a run-time value expand into conversion instructions, which
// this GPU issues to its FP64 pipe.  The twiddle index r k step stays below M
// (r < R, k < Ns, step = M / (Ns R)), so it needs no reduction.
template <int R>
__device__ __forceinline__ void fft_stage(const float4* x, float4* y, int MR, int Ns, int lgNs, int step,
                                          const float4* tw, int tws, int lane) {
    for (int j = lane; j < MR; j += 32) {
        const int jq = lgNs >= 0 ? (j >> lgNs) : j / Ns;
        const int k = j - jq * Ns;
        cff v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = ldc(x, j + r * MR);
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], ldc(tw, r * k * step * tws));
        }
        if (R == 2) {
            const cff a = v[0], b = v[1];
            v[0] = cadd(a, b);
            v[1] = csub(a, b);
        } else if (R == 4) {
            const cff t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
            const cff t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
            v[0] = cadd(t0, t2);
            v[2] = csub(t0, t2);
            v[1] = sub_i(t1, t3);
            v[3] = add_i(t1, t3);
        } else {
            // w = e^{-2 pi i/3}: a + w b + w^2 c = m - i s3 (b - c), m = a - (b + c)/2
            const cff a = v[0];
            const cff bc = cadd(v[1], v[2]), bmc = csub(v[1], v[2]);
            v[0] = cadd(a, bc);
            const cff m = cff{sub(a.re, mul_f(bc.re, 0.5f)), sub(a.im, mul_f(bc.im, 0.5f))};
            const ff s3{kS3Hi, kS3Lo};
            const cff sb = cff{mul(bmc.re, s3), mul(bmc.im, s3)};
            v[1] = sub_i(m, sb);
            v[2] = add_i(m, sb);
        }
        const int idxD = jq * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) stc(y, idxD + r * Ns, v[r]);
    }
}

// Warp Stockham FFT (forward) of M = 2^a 3^b complex float-float values in
// shared memory; x, y: buffers of M; tw[e * tws] = e^{-2 pi i e / M}.
// Returns the buffer holding the result.
__device__ float4* warp_fft_ff(float4* x, float4* y, int M, const float4* tw, int lane, int tws) {
    int rem = M, Ns = 1, lgNs = 0;
    while (rem > 1) {
        const int R = (rem & 3) == 0 ? 4 : ((rem & 1) == 0 ? 2 : 3);
        const int MR = M / R, step = M / (Ns * R);
        if (R == 4)
            fft_stage<4>(x, y, MR, Ns, lgNs, step, tw, tws, lane);
        else if (R == 2)
            fft_stage<2>(x, y, MR, Ns, lgNs, step, tw, tws, lane);
        else
            fft_stage<3>(x, y, MR, Ns, lgNs, step, tw, tws, lane);
        __syncwarp();
        float4* t = x;
        x = y;
        y = t;
        Ns *= R;
        lgNs = (lgNs >= 0 && R != 3) ? lgNs + (R == 4 ? 2 : 1) : -1;
        rem /= R;
    }
    return x;
}

__device__ __forceinline__ ff shfl_xor_ff(ff v, int o) {
    return ff{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ ff shfl_up_ff(ff v, int o) {
    return ff{__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o)};
}

// DFT of an even sequence x_0..x_{L-1} (x_k = x_{L-k}, L = 2K) from its K+1
// distinct values, in place (xh[0..K] -> X_0..X_K): the algorithm of
// warp_even_dft (kernels.cu) in float-float.  y, scr: K values of scratch;
// twL[e * tws] = e^{-2 pi i e / L}; hs[e * tws] = (1/2 + Im twL, 1/2 - Im twL)
// as two float pairs.
__device__ void warp_even_dft_ff(float4* xh, float4* y, float4* scr, int K, const float4* twL,
                                 const float4* hs, int tws, int lane) {
    cff part = czero();
    for (int j = lane; j < K; j += 32) {
        const cff a = ldc(xh, j), b = ldc(xh, K - j);
        const float4 t = twL[j * tws];
        const float4 h = hs[j * tws];
        const ff hx{h.x, h.y}, hy{h.z, h.w};
        stc(y, j, cff{dot2(a.re, hx, b.re, hy), dot2(a.im, hx, b.im, hy)});
        const ff ct{t.x, t.y};
        part.re = add(part.re, mul(a.re, ct));
        part.im = add(part.im, mul(a.im, ct));
    }
    for (int o = 16; o > 0; o >>= 1) {
        part.re = add(part.re, shfl_xor_ff(part.re, o));
        part.im = add(part.im, shfl_xor_ff(part.im, o));
    }
    const cff x0 = ldc(xh, 0), xK = ldc(xh, K);
    const cff X1 = cff{sub(mul_f(part.re, 2.0f), add(x0.re, xK.re)), sub(mul_f(part.im, 2.0f), add(x0.im, xK.im))};
    __syncwarp();
    float4* Z = warp_fft_ff(y, scr, K, twL, lane, 2 * tws);
    float4* I = (Z == y) ? scr : y;
    const int H = K / 2;
    for (int kk = lane; kk <= H; kk += 32) {
        const cff zk = ldc(Z, kk), zc = ldc(Z, kk == 0 ? 0 : K - kk);
        stc(xh, 2 * kk, cff{add(zk.re, zc.re), add(zk.im, zc.im)});
        stc(I, kk, cff{sub(zk.im, zc.im), sub(zc.re, zk.re)});
    }
    __syncwarp();
    // odd outputs: X_{2k+1} = X_1 - sum_{m=1}^{k} I_m, k = 0..H-1 (warp scan)
    const int per = (H + 31) / 32;
    const int b0 = lane * per;
    cff run = czero();
    for (int q = 0; q < per; ++q) {
        const int kk = b0 + q;
        if (kk >= 1 && kk < H) run = cadd(run, ldc(I, kk));
    }
    cff incl = run;
    for (int o = 1; o < 32; o <<= 1) {
        const cff v = cff{shfl_up_ff(incl.re, o), shfl_up_ff(incl.im, o)};
        if (lane >= o) incl = cadd(incl, v);
    }
    cff acc = csub(X1, csub(incl, run));
    for (int q = 0; q < per; ++q) {
        const int kk = b0 + q;
        if (kk >= H) break;
        if (kk >= 1) acc = csub(acc, ldc(I, kk));
        stc(xh, 2 * kk + 1, acc);
    }
    __syncwarp();
}

// Per-pair quantities of the float-float far kernel (one per warp), in units
// of L = 2^eL: d~^2 / L^2, rho~ rho~' / L^2, omega_r L, and the normal
// factors / L of both orientations.
struct FarPairFF {
    float4 d2, rr;
    float4 nd0, nds, nd0t, ndst;
    float2 wl[2];
    int eL, real;
    int pad[2];
};

struct FarArgsFF {
    DeviceTables T;
    int N, M, mode_lo, mode_hi;
    double w1, w2;
    float2 c4;      // (1 / 4 pi)(2 pi / M) = 1 / (2 M) as a float pair
    double2* A;     // [mode][col][row], ld 2N
    double2* raw;   // [mode][kernel][l][m]
};

__host__ __device__ __forceinline__ int far_ff_tile_m(int nw) { return nw >= 16 ? 4 : 2; }

__device__ __forceinline__ cff sin2_mode_ff(const float4* gh, int n) {
    const cff gn = ldc(gh, n), gm = ldc(gh, n == 0 ? 1 : n - 1), gp = ldc(gh, n + 1);
    // G_n / 2 - (G_{n-1} + G_{n+1}) / 4
    return cff{sub(mul_f(gn.re, 0.5f), mul_f(add(gm.re, gp.re), 0.25f)),
               sub(mul_f(gn.im, 0.5f), mul_f(add(gm.im, gp.im), 0.25f))};
}
__device__ __forceinline__ cff nd_mode_ff(cff nd0, cff nds, cff gn, cff s2, bool real) {
    if (real)
        return cff{dot2(nd0.re, gn.re, nds.re, s2.re), dot2(nd0.re, gn.im, nds.re, s2.im)};
    return cadd(cmul(nd0, gn), cmul(nds, s2));
}
// complex128 of f v 2^sh (f a float pair)
__device__ __forceinline__ double2 out_c128(cff v, ff f, int sh) {
    return make_double2(to_double(mul(v.re, f), sh), to_double(mul(v.im, f), sh));
}

__device__ __forceinline__ cff cff_of(double2 z, int sh) {
    return cff{from_double(ldexp(z.x, sh)), from_double(ldexp(z.y, sh))};
}

__global__ void __launch_bounds__(512, 1) far_kernel_ff(FarArgsFF a) {
    extern __shared__ float4 smf[];
    const int M = a.M, N = a.N, K = M / 2, S1 = K + 1;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int TM = far_ff_tile_m(nw), TL = nw / TM;
    const int l0 = blockIdx.x * TL, m0 = blockIdx.y * TM;
    if (l0 + TL - 1 < m0) return;
    float4* tw = smf;                                   // M
    float4* hs = tw + M;                                // K
    float4* cs = hs + K;                                // S1: (sin^2(psi/2), cos psi)
    float4* trig = cs + S1;                             // kTrigTab
    float2* expt = reinterpret_cast<float2*>(trig + kTrigTab);          // kExpTab
    FarPairFF* geo = reinterpret_cast<FarPairFF*>(trig + kTrigTab + kExpTab / 2);
    float4* bufs = reinterpret_cast<float4*>(geo + nw);  // per warp: 4 S1 + 2 K
    int* act = reinterpret_cast<int*>(bufs + (size_t)nw * (4 * S1 + 2 * K));
    int* emax = act + nw;                               // nw x 2
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const float4 t = a.T.twid_ff[i];
        tw[i] = t;
        if (i < K) {
            const ff im{t.z, t.w};
            const ff hx = add_f(im, 0.5f), hy = add_f(neg(im), 0.5f);
            hs[i] = make_float4(hx.hi, hx.lo, hy.hi, hy.lo);
        }
    }
    for (int i = threadIdx.x; i < S1; i += blockDim.x) cs[i] = a.T.cos_ff[i];
    for (int i = threadIdx.x; i < kTrigTab; i += blockDim.x) trig[i] = a.T.trig_ff[i];
    for (int i = threadIdx.x; i < kExpTab; i += blockDim.x) expt[i] = a.T.exp_ff[i];
    // Pair set-up in FP64, all pairs of the CTA by the lanes of warp 0 (lane
    // w: pair w): the FP64 pipe is 1/64 of the FP32 one and a warp
    // instruction occupies it whatever the number of active lanes, so one
    // lane per warp would cost nw times as much.
    if (warp == 0 && lane < nw) {
        const int wq = lane;
        const int l = l0 + wq % TL, m = m0 + wq / TL;
        int f = 0;
        if (l < N && m < N && l >= m) {
            f = 4;
            if (l > m) {
                f |= (a.T.cls[(size_t)l * N + m] == kFar ? 1 : 0) | (a.T.cls[(size_t)m * N + l] == kFar ? 2 : 0);
                if (f & 3) {
                    const PairGeom g = grid_pair(a.T, l, m);
                    const bool real = g.d2.y == 0.0 && g.rr.y == 0.0 && g.nd0.y == 0.0 && g.nds.y == 0.0 &&
                                      g.nd0t.y == 0.0 && g.ndst.y == 0.0;
                    if (real) f |= 8;
                    const double lsq = fabs(g.d2.x) + fabs(g.d2.y) + 4.0 * (fabs(g.rr.x) + fabs(g.rr.y));
                    const int eL = ilogb(lsq) / 2;
                    FarPairFF p;
                    p.d2 = pack(cff_of(g.d2, -2 * eL));
                    p.rr = pack(cff_of(g.rr, -2 * eL));
                    p.nd0 = pack(cff_of(g.nd0, -eL));
                    p.nds = pack(cff_of(g.nds, -eL));
                    p.nd0t = pack(cff_of(g.nd0t, -eL));
                    p.ndst = pack(cff_of(g.ndst, -eL));
                    const ff w1 = from_double(ldexp(a.w1, eL)), w2 = from_double(ldexp(a.w2, eL));
                    p.wl[0] = make_float2(w1.hi, w1.lo);
                    p.wl[1] = make_float2(w2.hi, w2.lo);
                    p.eL = eL;
                    p.real = real ? 1 : 0;
                    geo[wq] = p;
                }
            }
        }
        act[wq] = f;
    }
    __syncthreads();
    const Tables TT{expt, trig};

    // samples j = 0..K of the CTA's pairs over all threads (units of L):
    //   S'_j = e^{iq} / R',  G'_j = -/+ e^{iq} (1 - iq) / R'^3  (region a: -, b: +)
    // with e^{-Im q} = mantissa x 2^{E_j}; E_j kept in the scratch area
    // (pair w, angle j) over the CTA's threads; the index pair advances by
    // blockDim.x without a run-time division
    int w = threadIdx.x / S1, j = threadIdx.x - (threadIdx.x / S1) * S1;
    const int bstep = blockDim.x / S1, jstep = blockDim.x - bstep * S1;
    for (; w < nw; w += bstep, j += jstep) {
        if (j >= S1) {
            j -= S1;
            ++w;
            if (w >= nw) break;
        }
        if (!(act[w] & 3)) continue;
        const FarPairFF& p = geo[w];
        float4* buf = bufs + (size_t)w * (4 * S1 + 2 * K);
        int* Eb = reinterpret_cast<int*>(buf + 4 * S1);
        const float4 scv = cs[j];
        const ff s2x4 = mul_f(ff{scv.x, scv.y}, 4.0f);
        if (p.real) {
            const ff D2 = add(ff{p.d2.x, p.d2.y}, mul(ff{p.rr.x, p.rr.y}, s2x4));
            const ff iR = rsqrt(D2), R = mul(D2, iR);
            const ff gk = mul(sqr(iR), iR);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const ff q = mul(ff{p.wl[r].x, p.wl[r].y}, R);
                ff sn, cn;
                sincos_ff(q, TT, sn, cn);
                const cff S{mul(cn, iR), mul(sn, iR)};
                const ff gr = r == 0 ? neg(gk) : gk;
                const cff G{mul(gr, add(cn, mul(q, sn))), mul(gr, sub(sn, mul(q, cn)))};
                stc(buf, (2 * r) * S1 + j, S);
                stc(buf, (2 * r + 1) * S1 + j, G);
                Eb[r * S1 + j] = 0;
            }
            continue;
        }
        const cff D2 = cadd(unpack(p.d2), cscale(unpack(p.rr), s2x4));
        cff R, iR;
        csqrt_rcp(D2, R, iR);
        const cff gk = cmul(iR, cmul(iR, iR));
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const cff q = cscale(R, ff{p.wl[r].x, p.wl[r].y});
            int E;
            const ff mag = exp_split(neg(q.im), TT, E);
            ff sn, cn;
            sincos_ff(q.re, TT, sn, cn);
            const cff e{mul(mag, cn), mul(mag, sn)};
            const cff S = cmul(e, iR);
            const cff om{add_f(q.im, 1.0f), neg(q.re)};   // 1 - i q
            cff G = cmul(cmul(gk, e), om);
            if (r == 0) G = cneg(G);
            stc(buf, (2 * r) * S1 + j, S);
            stc(buf, (2 * r + 1) * S1 + j, G);
            Eb[r * S1 + j] = E;
        }
    }
    __syncthreads();
    // common exponent per (pair, medium), then the four transforms (per warp)
    if (act[warp] & 3) {
        float4* buf = bufs + (size_t)warp * (4 * S1 + 2 * K);
        const int* Eb = reinterpret_cast<const int*>(buf + 4 * S1);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            int em = -(1 << 30);
            for (int j = lane; j < S1; j += 32) em = max(em, Eb[r * S1 + j]);
            for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
            for (int j = lane; j < S1; j += 32) {
                const int d = Eb[r * S1 + j] - em;
                if (d == 0) continue;
                for (int s = 0; s < 2; ++s) {
                    const int i = (2 * r + s) * S1 + j;
                    buf[i] = d < -120 ? make_float4(0.f, 0.f, 0.f, 0.f) : pack(cldexp(ldc(buf, i), d));
                }
            }
            if (lane == 0) emax[2 * warp + r] = em;
        }
        __syncwarp();
        float4* y = buf + 4 * S1;
        for (int s = 0; s < 4; ++s) warp_even_dft_ff(buf + s * S1, y, y + K, K, tw, hs, 1, lane);
    }
    __syncthreads();

    // scatter: thread (pair w, mode n) writes the entries of both orientations
    const int nmodes = a.mode_hi - a.mode_lo;
    const int lg = __ffs(nw) - 1, lgl = __ffs(TL) - 1;
    const int total = nmodes << lg;
    const ff c4{a.c4.x, a.c4.y};
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int w = idx & (nw - 1), n = idx >> lg;
        const int f = act[w];
        if (!(f & 4)) continue;
        const int l = l0 + (w & (TL - 1)), m = m0 + (w >> lgl);
        const int nn = a.mode_lo + n;
        cff sa = czero(), sb = sa, ka[2] = {sa, sa}, kb[2] = {sa, sa};
        int shS[2] = {0, 0}, shK[2] = {0, 0};   // exponents of S^ and K^ per medium
        if (f & 3) {
            const float4* b = bufs + (size_t)w * (4 * S1 + 2 * K);
            const FarPairFF& p = geo[w];
            const bool real = p.real != 0;
            sa = ldc(b, nn);
            sb = ldc(b, 2 * S1 + nn);
            const cff ga = ldc(b, S1 + nn), gb = ldc(b, 3 * S1 + nn);
            const cff s2a = sin2_mode_ff(b + S1, nn), s2b = sin2_mode_ff(b + 3 * S1, nn);
            if (f & 1) {
                ka[0] = nd_mode_ff(unpack(p.nd0), unpack(p.nds), ga, s2a, real);
                kb[0] = nd_mode_ff(unpack(p.nd0), unpack(p.nds), gb, s2b, real);
            }
            if (f & 2) {
                ka[1] = nd_mode_ff(unpack(p.nd0t), unpack(p.ndst), ga, s2a, real);
                kb[1] = nd_mode_ff(unpack(p.nd0t), unpack(p.ndst), gb, s2b, real);
            }
            const int ea = real ? 0 : emax[2 * w], eb = real ? 0 : emax[2 * w + 1];
            shS[0] = ea - p.eL;
            shS[1] = eb - p.eL;
            shK[0] = ea - 2 * p.eL;
            shK[1] = eb - 2 * p.eL;
        }
        for (int o = 0; o < 2; ++o) {
            if (o == 1 && l == m) break;
            const int tgt = o == 0 ? l : m, src = o == 0 ? m : l;
            const bool on = (f >> o) & 1;
            const double2 z = make_double2(0.0, 0.0);
            if (a.A) {
                // blocks: K^a -> (t, s); -S^a -> (t, N+s); K^b -> (N+t, s); S^b -> (N+t, N+s)
                const size_t ld = 2 * (size_t)N;
                double2* col0 = a.A + (size_t)n * ld * ld + (size_t)src * ld;
                double2* col1 = col0 + (size_t)N * ld;
                if (on) {
                    const float2 fu = a.T.wuc_ff[src], fp = a.T.wpc_ff[src];
                    const ff wu{fu.x, fu.y}, wp{fp.x, fp.y};
                    col0[tgt] = out_c128(ka[o], wu, shK[0]);
                    col1[tgt] = out_c128(sa, neg(wp), shS[0]);
                    col0[N + tgt] = out_c128(kb[o], wu, shK[1]);
                    col1[N + tgt] = out_c128(sb, wp, shS[1]);
                } else {
                    col0[tgt] = z;
                    col1[tgt] = z;
                    col0[N + tgt] = z;
                    col1[N + tgt] = z;
                }
            }
            if (a.raw) {
                const size_t NN = (size_t)N * N, e = (size_t)tgt * N + src;
                a.raw[((size_t)n * 4 + 0) * NN + e] = on ? out_c128(sa, c4, shS[0]) : z;
                a.raw[((size_t)n * 4 + 1) * NN + e] = on ? out_c128(ka[o], c4, shK[0]) : z;
                a.raw[((size_t)n * 4 + 2) * NN + e] = on ? out_c128(sb, c4, shS[1]) : z;
                a.raw[((size_t)n * 4 + 3) * NN + e] = on ? out_c128(kb[o], c4, shK[1]) : z;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Close pairs, stage 2, in float-float (mixed path): the algorithm of
// near_modes_kernel (kernels.cu) -- split samples, even DFTs, FFT convolution
// with the exact modal Laplace kernels -- with the samples, transforms and
// convolution in FP32 pairs.  The Laplace kernels Z^_m, D^_m stay FP64 (the
// near-singular part of the split, stage 1) and enter the convolution scaled
// by a power of two each (their largest exponent).  Lengths are in units of
// L = 2^eL (L^2 ~ |d~^2| + 4 |rho~ rho~'|), e^{-Im q} is carried as mantissa x
// 2^E per sample and rescaled to a common exponent per medium before the
// transforms; the exponents return in the FP64 outputs.  Close pairs with a
// point in the PML (the Sec. 4.3 substitution, or the diagnostic exact split
// of subst_off) are left to the FP64 kernel.
// ---------------------------------------------------------------------------
struct NearArgsFF {
    const NearPair* np;
    const float4* pff;     // per-pair quantities (kNearFF float4 each), from the Laplace-mode kernel
    const float4* twid2;
    const float4* trig;
    const float2* expt;
    int npairs, M, L, mode_lo, mode_hi;
    double w1, w2;
    const double2* zd;     // [p][2][M]: Z^_m, D^_m (FP64)
    double2* out;          // [p][4][nmodes]
    float4 pa[8], pb[8];   // Taylor coefficients of cH1 (pa) and cH3 (pb)
    float2 scale;          // 2 pi / M
    float2 cconv;          // 1 / (2 pi 2M)
    float2 wq[2], wc[2];   // omega_r / (4 pi), omega_r^3 / (4 pi)
    float2 inv4pi;         // 1 / (4 pi)
    int share_mirror;      // 1: a packed grid pair and its mirror in one CTA
};

// x 2^-shift as a float pair, with 32-bit integer operations only (x normal
// and the result in float's normal range; zero, denormal or tiny results
// give 0): hi = the significand's top 24 bits rounded, lo = the remaining 29
// bits (signed) as a float, both with x's exponent.
__device__ __forceinline__ ff ff_of_double(double x, int shift) {
    const uint32_t whi = (uint32_t)__double2hiint(x), wlo = (uint32_t)__double2loint(x);
    const int e = (int)((whi >> 20) & 0x7ffu);
    const int ee = e - 1023 - shift;
    if (e == 0 || ee < -74) return ff{0.0f, 0.0f};
    if (ee > 126) return ff{__int_as_float(0x7f800000), 0.0f};
    // 53-bit significand m = (mh: bits 32..52, wlo): top 24 bits rounded
    const uint32_t mh = (whi & 0xfffffu) | 0x100000u;        // bits 32..52
    // m >> 29 = (mh << 3) | (wlo >> 29); round with bit 28
    uint32_t top = (mh << 3) | (wlo >> 29);
    const uint32_t rest = wlo & 0x1fffffffu;                  // bits 0..28
    int r;                                                    // m - (top << 29) after rounding, |r| <= 2^28
    if (rest & 0x10000000u) {
        top += 1u;
        r = (int)rest - (int)0x20000000u;
    } else {
        r = (int)rest;
    }
    int eh = ee;
    if (top >> 24) {
        top >>= 1;
        eh += 1;
    }
    const uint32_t sg = whi & 0x80000000u;
    const float hi = __uint_as_float(sg | ((uint32_t)(eh + 127) << 23) | (top & 0x7fffffu));
    float lo = __int2float_rn(r) * __int_as_float((ee - 52 + 127) << 23);
    if (sg) lo = -lo;
    return ff{hi, lo};
}
__device__ __forceinline__ cff cff_of_double(double2 z, int shift) {
    return cff{ff_of_double(z.x, shift), ff_of_double(z.y, shift)};
}
// largest binary exponent of |x| (integer operations; -2000 for zero)
__device__ __forceinline__ int exp_of_double(double x) {
    const int e = (int)(((uint32_t)__double2hiint(x) >> 20) & 0x7ffu);
    return e == 0 ? -2000 : e - 1023;
}

// (sin q - q cos q) / q^3 for real q: the series to q^12 below |q| = 1/2, else
// the closed form (whose cancellation costs ~3/q^2 ulps)
__device__ __forceinline__ ff h4_ff(ff q, ff sn, ff cs, ff iq) {
    if (fabsf(q.hi) < 0.5f) {
        const ff q2 = sqr(q);
        // 1/3 - q^2/30 + q^4/840 - q^6/45360 + q^8/3991680 - q^10/518918400 + q^12/93405312000
        const float x = q2.hi;
        float t = __fmaf_rn(x, 1.0f / 93405312000.0f, -1.0f / 518918400.0f);
        t = __fmaf_rn(x, t, 1.0f / 3991680.0f);
        t = __fmaf_rn(x, t, -1.0f / 45360.0f);
        t = __fmaf_rn(x, t, 1.0f / 840.0f);
        // 1/3 - q^2/30 + q^4 t in float-float for the first two terms
        ff v = mul_f(q2, -1.0f / 30.0f);
        v = add(v, ff{0x1.555556p-2f, -0x1.555556p-27f});   // 1/3
        return add_f(v, x * x * t);
    }
    const ff num = sub(sn, mul(q, cs));
    return mul(num, mul(sqr(iq), iq));
}

// sum_{k = k0}^{L} c_k q^{k - k0} (Horner; L <= 7)
__device__ __forceinline__ cff cpoly_ff(const float4 (&c)[8], int k0, int L, cff q) {
    cff r = czero();
#pragma unroll
    for (int k = 7; k >= 0; --k)
        if (k >= k0 && k <= L) r = cadd(cmul(r, q), unpack(c[k]));
    return r;
}

// Close-pair modes in float-float (pairs without a PML point; the others
// return at once).  Mirror sharing (a.share_mirror) for packed pairs: a grid
// pair (l, m) and its mirror (m, l) share R(psi), the f1, r1, f3 samples and
// spectra, Z^ and the S^ results; the CTA of the lower index adds the mirror's
// double-layer remainder r3 (its own normal factor N_D) and its transform, the
// mirror's D^ transform and one product and inverse transform, and writes both
// pairs' modes; the mirror's CTA returns.  The mirror's buffers: its D^ and K
// convolution (2 x (M+1)), its r3 spectrum (K+1), and a third 2M scratch slot
// in the region-b sample sequences, which packed pairs do not use.
__global__ void __launch_bounds__(128) near_modes_kernel_ff(NearArgsFF a) {
    extern __shared__ float4 smf[];
    const int M = a.M, K = M / 2, S1 = K + 1, L2 = 2 * M, S2 = M + 1, p = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* tw2 = smf;                  // 2M: e^{-2 pi i e / (2M)}
    float4* hs = tw2 + L2;              // M: even-DFT weights
    float4* seq = hs + M;               // 8 sequences of S1
    float4* cv = seq + 8 * S1;          // 4 sequences of S2
    float4* slots = cv + 4 * S2;        // 2 slots of 2M
    float4* trig = slots + 4 * M;       // kTrigTab
    float2* expt = reinterpret_cast<float2*>(trig + kTrigTab);   // kExpTab
    int* Eb = reinterpret_cast<int*>(trig + kTrigTab + kExpTab / 2);   // 2 x S1
    int* ex = Eb + 2 * S1;              // [0..1] common sample exponent per medium, [2] eZ, [3] eD, [4] the mirror's eD
    // mirror sharing: S2 + S2 + S1, from the first 16-byte boundary after Eb
    // and ex[0..4] (Eb itself starts on one)
    float4* zDm = reinterpret_cast<float4*>(Eb) + (2 * S1 + 5 + 3) / 4;
    float4* cKm = zDm + S2;
    float4* seqm = cKm + S2;
    float4* slot2 = seq + 4 * S1;       // 2M <= 4 (K + 1): region b's sequences (unused by packed pairs)
    float4* slot = slots + (warp & 1) * 2 * M;
    float4* wyK = slot + (warp >> 1) * M;
    for (int i = threadIdx.x; i < L2; i += blockDim.x) {
        const float4 t = a.twid2[i];
        tw2[i] = t;
        if (i < M) {
            const ff im{t.z, t.w};
            const ff hx = add_f(im, 0.5f), hy = add_f(neg(im), 0.5f);
            hs[i] = make_float4(hx.hi, hx.lo, hy.hi, hy.lo);
        }
    }
    for (int i = threadIdx.x; i < kTrigTab; i += blockDim.x) trig[i] = a.trig[i];
    for (int i = threadIdx.x; i < kExpTab; i += blockDim.x) expt[i] = a.expt[i];
    if (threadIdx.x < 5) ex[threadIdx.x] = threadIdx.x < 2 ? 0 : -2000;
    const NearPair& q = a.np[p];
    const bool plain = (q.flags & kFlagFar) != 0;
    const bool subst = (q.flags & kFlagSubst) != 0;
    // Pairs with a point in the PML take the FP64 kernel: their split's two
    // terms (the polynomial of the Sec. 4.3 substitution grows like |2q|^L /
    // L!) cancel by up to ~1e10 at |q| ~ 100, beyond a float pair's 48 bits.
    if (subst) return;
    // pair quantities in units of L = 2^eL, computed in FP64 by the Laplace-
    // mode kernel (one pair per thread there: the FP64 pipe is 1/64 of the
    // FP32 one and a warp instruction occupies it whatever its active lanes)
    const float4* pf = a.pff + (size_t)p * kNearFF;
    const int L = a.L;
    __syncthreads();
    const float4 misc = pf[6];
    const bool packed = !plain && __float_as_int(misc.y) != 0;
    const int eL = __float_as_int(misc.x);
    const cff d2 = unpack(pf[0]), rr = unpack(pf[1]), nd0 = unpack(pf[2]), nds = unpack(pf[3]);
    // mirror sharing (both pairs packed: physical, not far, no substitution;
    // their units 2^eL agree, |d~^2| + 4 |rho~ rho~'| being symmetric)
    bool share = false;
    cff nd0m = czero(), ndsm = czero();
    if (a.share_mirror && packed && q.mirror >= 0) {
        const NearPair& qm = a.np[q.mirror];
        const float4* pfm = a.pff + (size_t)q.mirror * kNearFF;
        share = (qm.flags & (kFlagFar | kFlagSubst)) == 0 && __float_as_int(pfm[6].y) != 0;
        if (share && q.mirror < p) return;    // computed by the mirror's CTA (uniform)
        if (share) {
            nd0m = unpack(pfm[2]);
            ndsm = unpack(pfm[3]);
        }
    }
    const float4 wv = pf[4], iwv = pf[5];
    const ff wl[2] = {ff{wv.x, wv.y}, ff{wv.z, wv.w}};
    const ff iwl[2] = {ff{iwv.x, iwv.y}, ff{iwv.z, iwv.w}};
    const ff wq[2] = {ff{a.wq[0].x, a.wq[0].y}, ff{a.wq[1].x, a.wq[1].y}};
    const ff wc[2] = {ff{a.wc[0].x, a.wc[0].y}, ff{a.wc[1].x, a.wc[1].y}};
    const ff inv4pi{a.inv4pi.x, a.inv4pi.y};
    const Tables TT{expt, trig};
    for (int j = threadIdx.x; j <= K; j += blockDim.x) {
        // sin^2(psi_j / 2) from the length-2M twiddles: psi_j / 2 = pi j / M = 2 pi j / (2M)
        const float4 tj = tw2[j];
        const ff sj{-tj.z, -tj.w};                  // sin(pi j / M)
        const ff s2 = sqr(sj);
        const ff s2x4 = mul_f(s2, 4.0f);
        if (packed) {
            // D2 >= 2^-120: below it (a correction point next to its target in
            // a graded cluster, at j = 0) the samples are their q -> 0 limits
            ff D2 = add(d2.re, mul(rr.re, s2x4));
            if (D2.hi < 0x1p-120f) D2 = ff{0x1p-120f, 0.0f};
            const ff iR = rsqrt(D2), R = mul(D2, iR);
            const ff ND = add(nd0.re, mul(nds.re, s2));
            const ff NDm = add(nd0m.re, mul(ndsm.re, s2));
            ff f1[2], r1[2], f3[2], r3[2], r3m[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const ff qr = mul(wl[r], R), iq = mul(iR, iwl[r]);
                ff sn, cs;
                sincos_ff(qr, TT, sn, cs);
                f1[r] = cs;
                r1[r] = mul(wq[r], mul(sn, iq));
                f3[r] = add(cs, mul(qr, sn));
                const ff h4w = mul(wc[r], h4_ff(qr, sn, cs, iq));
                r3[r] = mul(h4w, r == 0 ? neg(ND) : ND);
                r3m[r] = mul(h4w, r == 0 ? neg(NDm) : NDm);
            }
            stc(seq, 0 * S1 + j, cff{f1[0], f1[1]});
            stc(seq, 1 * S1 + j, cff{r1[0], r1[1]});
            stc(seq, 2 * S1 + j, cff{f3[0], f3[1]});
            stc(seq, 3 * S1 + j, cff{r3[0], r3[1]});
            if (share) stc(seqm, j, cff{r3m[0], r3m[1]});
            continue;
        }
        const cff D2 = cadd(d2, cscale(rr, s2x4));
        cff R, iR;
        csqrt_rcp(D2, R, iR);
        const cff ND = cadd(nd0, cscale(nds, s2));
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const cff qq = cscale(R, wl[r]);
            int E;
            const ff mag = exp_split(neg(qq.im), TT, E);
            ff sn, cs;
            sincos_ff(qq.re, TT, sn, cs);
            const cff e{mul(mag, cs), mul(mag, sn)};
            cff v0, v1, v2, v3;
            if (plain) {
                // S~ = e / (4 pi R) (x 2^-eL); K~ = -sg N_D e (1 - iq) / (4 pi R^3) (x 2^-2eL)
                v0 = cscale(cmul(e, iR), inv4pi);
                const cff iR3 = cmul(iR, cmul(iR, iR));
                cff Dk = cscale(cmul(ND, iR3), inv4pi);
                if (r == 0) Dk = cneg(Dk);
                v2 = cmul(cmul(Dk, e), cff{add_f(qq.im, 1.0f), neg(qq.re)});
                v1 = czero();
                v3 = czero();
            } else {
                // cH1 = e P_a(q), Z (e^{iq} - cH1) = -(w / 4 pi) e sum_{k>=1} a_k q^{k-1};
                // cH3 = e P_b(q), D (e^{iq}(1 - iq) - cH3) = (w^3 / 4 pi) N_D e sum_{k>=3} b_k q^{k-3}
                const cff pa1 = cpoly_ff(a.pa, 1, L, qq);
                const cff pa0 = cadd(unpack(a.pa[0]), cmul(qq, pa1));
                const cff pb3 = cpoly_ff(a.pb, 3, L, qq);
                cff pb0 = cadd(unpack(a.pb[2]), cmul(qq, pb3));
                pb0 = cadd(unpack(a.pb[1]), cmul(qq, pb0));
                pb0 = cadd(unpack(a.pb[0]), cmul(qq, pb0));
                v0 = cmul(e, pa0);
                v1 = cscale(cmul(e, pa1), neg(wq[r]));
                v2 = cmul(e, pb0);
                v3 = cscale(cmul(cmul(ND, e), pb3), r == 0 ? wc[r] : neg(wc[r]));
            }
            stc(seq, (4 * r + 0) * S1 + j, v0);
            stc(seq, (4 * r + 1) * S1 + j, v1);
            stc(seq, (4 * r + 2) * S1 + j, v2);
            stc(seq, (4 * r + 3) * S1 + j, v3);
            Eb[r * S1 + j] = E;
        }
    }
    __syncthreads();
    // common exponent per medium (warps 0, 1), the Laplace kernels' exponents
    // (warps 2, 3)
    const int nmodes = a.mode_hi - a.mode_lo;
    const double2* Z = a.zd + (size_t)p * 2 * M;
    const double2* Dd = Z + M;
    if (!packed && warp < 2) {
        const int r = warp;
        int em = -(1 << 30);
        for (int j = lane; j < S1; j += 32) em = max(em, Eb[r * S1 + j]);
        for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
        for (int j = lane; j < S1; j += 32) {
            const int d = Eb[r * S1 + j] - em;
            if (d == 0) continue;
            for (int k = 0; k < 4; ++k) {
                const int i = (4 * r + k) * S1 + j;
                seq[i] = d < -120 ? make_float4(0.f, 0.f, 0.f, 0.f) : pack(cldexp(ldc(seq, i), d));
            }
        }
        if (lane == 0) ex[r] = em;
    }
    const double2* Ddm = share ? a.zd + (size_t)q.mirror * 2 * M + M : nullptr;
    if (!plain && (warp >= 2 || (share && warp == 0))) {
        const double2* X = warp == 2 ? Z : warp == 3 ? Dd : Ddm;
        int em = -2000;
        for (int i = lane; i <= M - 2; i += 32) em = max(em, max(exp_of_double(X[i].x), exp_of_double(X[i].y)));
        for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
        if (lane == 0) ex[warp == 0 ? 4 : warp] = em;
    }
    __syncthreads();
    // even-sequence DFTs of length M: packed pairs 4 (+ the mirror's r3),
    // plain pairs 0, 2, 4, 6, the others all 8
    if (packed) {
        warp_even_dft_ff(seq + warp * S1, wyK, wyK + K, K, tw2, hs, 2, lane);
        if (share && warp == 0) warp_even_dft_ff(seqm, wyK, wyK + K, K, tw2, hs, 2, lane);
    } else {
        for (int s = warp; s < 8; s += 4) {
            if (plain && (s & 1)) continue;
            warp_even_dft_ff(seq + s * S1, wyK, wyK + K, K, tw2, hs, 2, lane);
        }
    }
    __syncthreads();
    const ff scale{a.scale.x, a.scale.y}, cc{a.cconv.x, a.cconv.y};
    double2* out = a.out + (size_t)p * 4 * nmodes;
    if (plain) {
        for (int t = threadIdx.x; t < nmodes; t += blockDim.x) {
            const int n = a.mode_lo + t;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int r = k >> 1;
                const int sh = ex[r] - ((k & 1) ? 2 * eL : eL);
                out[(size_t)k * nmodes + t] = out_c128(ldc(seq, (2 * k) * S1 + n), scale, sh);
            }
        }
        return;
    }
    const int eZ = ex[2], eD = ex[3], eDm = ex[4];
    float4* zZ = cv;
    float4* zD = cv + S2;
    float4* cS = cv + 2 * S2;
    float4* cK = cv + 3 * S2;
    double2* outm = share ? a.out + (size_t)q.mirror * 4 * nmodes : nullptr;
    for (int i = threadIdx.x; i <= M; i += blockDim.x) {
        const bool inz = i <= M - 2;
        stc(zZ, i, inz ? cff_of_double(Z[i], eZ) : czero());
        stc(zD, i, inz ? cff_of_double(Dd[i], eD) : czero());
        if (share) stc(zDm, i, inz ? cff_of_double(Ddm[i], eDm) : czero());
    }
    __syncthreads();
    if (warp < 2) warp_even_dft_ff(warp == 0 ? zZ : zD, slot, slot + M, M, tw2, hs, 1, lane);
    if (share && warp == 2) warp_even_dft_ff(zDm, slot2, slot2 + M, M, tw2, hs, 1, lane);
    const int passes = packed ? 1 : 2;
    for (int r = 0; r < passes; ++r) {
        for (int i = threadIdx.x; i <= M; i += blockDim.x) {
            cff vS = czero(), vK = czero();
            if (i <= K - 1) {
                vS = cscale(ldc(seq, (packed ? 0 : 4 * r + 0) * S1 + i), scale);
                vK = cscale(ldc(seq, (packed ? 2 : 4 * r + 2) * S1 + i), scale);
                if (packed) vK.im = neg(vK.im);
            }
            stc(cS, i, vS);
            stc(cK, i, vK);
        }
        __syncthreads();
        if (warp >= 2) warp_even_dft_ff(warp == 2 ? cS : cK, slot, slot + M, M, tw2, hs, 1, lane);
        __syncthreads();
        for (int i = threadIdx.x; i <= M; i += blockDim.x) {
            stc(cS, i, cmul(ldc(zZ, i), ldc(cS, i)));
            const cff kh = ldc(cK, i);
            const cff k = cmul(ldc(zD, i), kh);
            stc(cK, i, r == 0 ? k : cneg(k));   // region b: D^ -> -D^ (unpacked)
            if (share) stc(cKm, i, cmul(ldc(zDm, i), kh));   // packed: one pass (r = 0)
        }
        __syncthreads();
        if (warp >= 2) warp_even_dft_ff(warp == 2 ? cS : cK, slot, slot + M, M, tw2, hs, 1, lane);
        if (share && warp == 1) warp_even_dft_ff(cKm, slot2, slot2 + M, M, tw2, hs, 1, lane);
        __syncthreads();
        for (int t = threadIdx.x; t < nmodes; t += blockDim.x) {
            const int n = a.mode_lo + t;
            const cff s0 = cscale(ldc(cS, n), cc), k0 = cscale(ldc(cK, n), cc);
            if (packed) {
                // real parts from the convolutions, imaginary parts from the remainders
                const cff rs = cscale(ldc(seq, 1 * S1 + n), scale), rk = cscale(ldc(seq, 3 * S1 + n), scale);
                const double2 sa = make_double2(to_double(s0.re, eZ), to_double(rs.re, 0));
                const double2 sb = make_double2(to_double(s0.im, eZ), to_double(rs.im, 0));
                out[0 * (size_t)nmodes + t] = sa;
                out[1 * (size_t)nmodes + t] = make_double2(to_double(k0.re, eD), to_double(rk.re, eL));
                out[2 * (size_t)nmodes + t] = sb;
                out[3 * (size_t)nmodes + t] = make_double2(to_double(k0.im, eD), to_double(rk.im, eL));
                if (share) {
                    const cff km = cscale(ldc(cKm, n), cc), rkm = cscale(ldc(seqm, n), scale);
                    outm[0 * (size_t)nmodes + t] = sa;
                    outm[1 * (size_t)nmodes + t] = make_double2(to_double(km.re, eDm), to_double(rkm.re, eL));
                    outm[2 * (size_t)nmodes + t] = sb;
                    outm[3 * (size_t)nmodes + t] = make_double2(to_double(km.im, eDm), to_double(rkm.im, eL));
                }
            } else {
                const int em = ex[r];
                const cff rs = cscale(ldc(seq, (4 * r + 1) * S1 + n), scale);
                const cff rk = cscale(ldc(seq, (4 * r + 3) * S1 + n), scale);
                out[(2 * r + 0) * (size_t)nmodes + t] =
                    make_double2(to_double(s0.re, eZ + em) + to_double(rs.re, em),
                                 to_double(s0.im, eZ + em) + to_double(rs.im, em));
                out[(2 * r + 1) * (size_t)nmodes + t] =
                    make_double2(to_double(k0.re, eD + em) + to_double(rk.re, em + eL),
                                 to_double(k0.im, eD + em) + to_double(rk.im, em + eL));
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Self-test of the float-float elementary functions (pmlbie_selftest_elementary
// selectors 20-22): exp as mantissa x 2^E, sin / cos, 1/sqrt of the float
// pair nearest to each double, returned as doubles.
// ---------------------------------------------------------------------------
__global__ void ff_elementary_kernel(int fn, const double* x, double* out, size_t n, const float2* exp_tab,
                                     const float4* trig_tab) {
    __shared__ float4 trig[kTrigTab];
    __shared__ float2 expt[kExpTab];
    for (int i = threadIdx.x; i < kTrigTab; i += blockDim.x) trig[i] = trig_tab[i];
    for (int i = threadIdx.x; i < kExpTab; i += blockDim.x) expt[i] = exp_tab[i];
    __syncthreads();
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Tables TT{expt, trig};
    const ff v = from_double(x[i]);
    if (fn == 20) {
        int E;
        const ff m = exp_split(v, TT, E);
        out[i] = to_double(m, E);
    } else if (fn == 21) {
        ff s, c;
        sincos_ff(v, TT, s, c);
        out[2 * i] = to_double(s, 0);
        out[2 * i + 1] = to_double(c, 0);
    } else if (fn == 22) {
        out[i] = to_double(rsqrt(v), 0);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void ff_tables(int M, std::vector<float4>& twid, std::vector<float4>& twid2, std::vector<float4>& cosv,
               std::vector<float2>& expv, std::vector<float4>& trig) {
    const double pi = 3.14159265358979323846;
    auto f2 = [](double x) {
        const float hi = (float)x;
        return make_float2(hi, (float)(x - (double)hi));
    };
    auto f4 = [&](double x, double y) {
        const float2 a = f2(x), b = f2(y);
        return make_float4(a.x, a.y, b.x, b.y);
    };
    twid.resize(M);
    twid2.resize(2 * M);
    cosv.resize(M / 2 + 1);
    for (int e = 0; e < M; ++e) twid[e] = f4(std::cos(2.0 * pi * e / M), -std::sin(2.0 * pi * e / M));
    for (int e = 0; e < 2 * M; ++e) twid2[e] = f4(std::cos(pi * e / M), -std::sin(pi * e / M));
    for (int j = 0; j <= M / 2; ++j) {
        const double s = std::sin(pi * j / M);
        cosv[j] = f4(s * s, std::cos(2.0 * pi * j / M));
    }
    expv.resize(kExpTab);
    for (int j = 0; j < kExpTab; ++j) expv[j] = f2(std::exp2(j / 64.0));
    trig.resize(kTrigTab);
    for (int k = 0; k < kTrigTab; ++k) trig[k] = f4(std::cos(pi * k / 256.0), std::sin(pi * k / 256.0));
}

// shared memory of a far_kernel_ff CTA with nw pairs
static size_t far_ff_smem(int M, int nw) {
    const size_t K = M / 2, S1 = K + 1;
    return sizeof(float4) * ((size_t)M + K + S1 + kTrigTab + kExpTab / 2 + (size_t)nw * (4 * S1 + 2 * K)) +
           sizeof(FarPairFF) * (size_t)nw + sizeof(int) * 3 * (size_t)nw;
}

bool far_ff_supported(const pmlbie_problem* prob) {
    // sin / cos of the float-float kernel take |q| < 2^16 pi/256: bound |q| by
    // max(omega) x (2 max |rho~| + z range) (every |dr| of the problem)
    const HostTables& H = prob->H;
    double rmax = 0.0, zmin = 0.0, zmax = 0.0;
    for (size_t i = 0; i < H.rho.size(); ++i) {
        rmax = std::max(rmax, std::abs(H.rho_t[i]));
        zmin = std::min(zmin, H.z[i]);
        zmax = std::max(zmax, H.z[i]);
    }
    const double qmax = std::max(prob->P.k1, prob->P.k2) * (2.0 * rmax + (zmax - zmin));
    return qmax < 780.0 && prob->D.twid_ff != nullptr;
}

static std::mutex g_far_ff_tune_mu;
static std::map<std::tuple<int, int, int, int>, int> g_far_ff_tuned;
// device time of the chosen configuration in its tuning launch (alone on the GPU)
static std::map<std::tuple<int, int, int, int>, float> g_far_ff_tuned_ms;

float far_ff_alone_ms(const pmlbie_problem* prob, int modes, bool raw) {
    std::lock_guard<std::mutex> lk(g_far_ff_tune_mu);
    auto it = g_far_ff_tuned_ms.find(std::make_tuple(prob->P.N, prob->P.M, modes, raw ? 1 : 0));
    return it == g_far_ff_tuned_ms.end() ? 0.f : it->second;
}

cudaError_t launch_far_ff(const pmlbie_problem* prob, const FarLaunch& fl, cudaStream_t s) {
    const int N = prob->P.N, M = prob->P.M;
    FarArgsFF a;
    a.T = prob->D;
    a.N = N;
    a.M = M;
    a.mode_lo = fl.mode_lo;
    a.mode_hi = fl.mode_hi;
    a.w1 = prob->P.k1;
    a.w2 = prob->P.k2;
    {
        const double c4 = 0.5 / M;
        const float hi = (float)c4;
        a.c4 = make_float2(hi, (float)(c4 - (double)hi));
    }
    a.A = fl.A;
    a.raw = fl.raw;
    cudaError_t e = allow_max_smem(far_kernel_ff);
    if (e != cudaSuccess) return e;
    auto run = [&](int nw) {
        g_far_pairs_per_cta = nw;
        const int tm = far_ff_tile_m(nw), tl = nw / tm;
        dim3 grid((N + tl - 1) / tl, (N + tm - 1) / tm);
        far_kernel_ff<<<grid, 32 * nw, far_ff_smem(M, nw), s>>>(a);
        count_launch();
        return cudaGetLastError();
    };
    const auto key = std::make_tuple(N, M, fl.mode_hi - fl.mode_lo, fl.raw ? 1 : 0);
    int nw = 0;
    {
        std::lock_guard<std::mutex> lk(g_far_ff_tune_mu);
        auto it = g_far_ff_tuned.find(key);
        if (it != g_far_ff_tuned.end()) nw = it->second;
    }
    if (nw) return run(nw);
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    if (!fl.tune) {
        for (int c : {8, 4, 2})
            if (far_ff_smem(M, c) <= (size_t)optin) return run(c);
        return cudaErrorInvalidConfiguration;
    }
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    int best = 0;
    float tbest = 1e30f;
    for (int c : {2, 4, 8, 16}) {
        if (far_ff_smem(M, c) > (size_t)optin) continue;
        float ms = 0.f;
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess || (e = run(c)) != cudaSuccess ||
            (e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
            break;
        if (ms < tbest) tbest = ms, best = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    if (!best) return cudaErrorInvalidConfiguration;
    std::lock_guard<std::mutex> lk(g_far_ff_tune_mu);
    g_far_ff_tuned[key] = best;
    g_far_ff_tuned_ms[key] = tbest;
    g_far_pairs_per_cta = best;
    return cudaSuccess;
}

cudaError_t launch_near_modes_ff(const pmlbie_problem* prob, int mode_lo, int mode_hi, const double2* zd,
                                 const float4* pff, double2* out, cudaStream_t s) {
    const int M = prob->P.M;
    NearArgsFF a;
    a.np = prob->D.near;
    a.pff = pff;
    a.twid2 = prob->D.twid2_ff;
    a.trig = prob->D.trig_ff;
    a.expt = prob->D.exp_ff;
    a.npairs = (int)prob->H.near.size();
    a.M = M;
    a.L = prob->P.taylor_L;
    a.mode_lo = mode_lo;
    a.mode_hi = mode_hi;
    a.w1 = prob->P.k1;
    a.w2 = prob->P.k2;
    a.zd = zd;
    a.out = out;
    double2 pa[8], pb[8];
    taylor_coeffs(a.L, pa, pb);
    auto f2 = [](double x) {
        const float hi = (float)x;
        return make_float2(hi, (float)(x - (double)hi));
    };
    for (int k = 0; k < 8; ++k) {
        const float2 ar = f2(pa[k].x), ai = f2(pa[k].y), br = f2(pb[k].x), bi = f2(pb[k].y);
        a.pa[k] = make_float4(ar.x, ar.y, ai.x, ai.y);
        a.pb[k] = make_float4(br.x, br.y, bi.x, bi.y);
    }
    const double i4p = 0.079577471545947667884;
    a.wq[0] = f2(a.w1 * i4p);
    a.wq[1] = f2(a.w2 * i4p);
    a.wc[0] = f2(a.w1 * a.w1 * a.w1 * i4p);
    a.wc[1] = f2(a.w2 * a.w2 * a.w2 * i4p);
    a.inv4pi = f2(i4p);
    a.scale = f2(2.0 * 3.14159265358979323846 / M);
    a.cconv = f2(1.0 / (2.0 * 3.14159265358979323846 * 2 * M));
    if (a.npairs == 0) return cudaSuccess;
    const size_t S1 = M / 2 + 1, S2 = M + 1;
    // ... + Eb (2 S1 ints) and ex (5 ints), rounded up to whole 16-byte units
    size_t smem = sizeof(float4) * (2 * (size_t)M + M + 8 * S1 + 4 * S2 + 4 * (size_t)M + kTrigTab + kExpTab / 2 +
                                    (2 * S1 + 5 + 3) / 4);
    // mirror sharing: the mirror's D^ and K convolution, its r3 spectrum
    const size_t share_bytes = sizeof(float4) * (2 * S2 + S1);
    a.share_mirror = smem + share_bytes <= 227 * 1024 ? 1 : 0;
    if (a.share_mirror) smem += share_bytes;
    cudaError_t e = allow_max_smem(near_modes_kernel_ff);
    if (e != cudaSuccess) return e;
    near_modes_kernel_ff<<<a.npairs, 128, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

bool ff_elementary_known(int fn) { return fn == 20 || fn == 21 || fn == 22; }

cudaError_t launch_ff_elementary(int fn, const double* x, double* out, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    std::vector<float4> tw, tw2, cv, trig;
    std::vector<float2> ex;
    ff_tables(8, tw, tw2, cv, ex, trig);
    float2* dexp = nullptr;
    float4* dtrig = nullptr;
    cudaError_t e = cudaMalloc(&dexp, sizeof(float2) * ex.size());
    if (e == cudaSuccess) e = cudaMalloc(&dtrig, sizeof(float4) * trig.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(dexp, ex.data(), sizeof(float2) * ex.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtrig, trig.data(), sizeof(float4) * trig.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        ff_elementary_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(fn, x, out, n, dexp, dtrig);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (dexp) cudaFree(dexp);
    if (dtrig) cudaFree(dtrig);
    return e;
}

}  // namespace pmlbie
