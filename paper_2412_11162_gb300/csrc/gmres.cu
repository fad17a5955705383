// Flexible GMRES refinement of the mixed-precision solve (not in the paper):
// for modes whose plain iterative refinement does not converge (condition
// number x FP32 LU error above 1), A x = B is solved by restarted FGMRES in
// FP64, right-preconditioned by the FP32 LU factors (Saad's flexible GMRES,
// the preconditioned vectors z_j = M^{-1} v_j are kept):
//
//   r = B - A x, v_0 = r/|r|;  for j: z_j = (L U)^{-1} v_j (FP32 triangular
//   solves; the flexible variant keeps the z_j actually computed), w = A z_j,
//   w <- w - V (V^H w) twice (classical Gram-Schmidt with reorthogonalisation),
//   h_{j+1,j} = |w|, v_{j+1} = w / h_{j+1,j}; complex Givens rotations keep
//   the least-squares residual |g_{j+1}|;  x <- x + Z y, H y = g.
//
// One instance per (mode, right-hand side); vectors are laid out like the
// solves, [mode][row][rhs], with one such array per Krylov vector.  Modes
// whose active flag is 0 are skipped by every kernel.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace pmlbie {

namespace {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) b
__device__ __forceinline__ double2 cdotm(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

constexpr int kRed = 256;

// block-wide sum of a double2 (kRed threads)
__device__ double2 block_sum(double2 v, double2* sh) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffff, v.x, o);
        v.y += __shfl_xor_sync(0xffffffff, v.y, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
    if (threadIdx.x < 32) {
        s = threadIdx.x < kRed / 32 ? sh[threadIdx.x] : make_double2(0.0, 0.0);
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffff, s.x, o);
            s.y += __shfl_xor_sync(0xffffffff, s.y, o);
        }
    }
    return s;   // valid in thread 0
}

// Y += A X over one chunk of kMvCols columns per CTA (Y zeroed first), grid
// (row blocks, column chunks, matrices): one active matrix spreads over many
// SMs ([b][n][nrhs] vectors, A column-major)
constexpr int kMvCols = 32;
__global__ void matvec_kernel(int n, int nrhs, const double2* A, const double2* X, double2* Y, const int* active) {
    const int b = blockIdx.z;
    if (active && !active[b]) return;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * nrhs) return;
    const int r = (int)(idx % nrhs), row = (int)(idx / nrhs);
    const int c0 = blockIdx.y * kMvCols, c1 = min(n, c0 + kMvCols);
    const double2* a = A + (size_t)b * n * n;
    const double2* x = X + (size_t)b * n * nrhs;
    double2 acc = make_double2(0.0, 0.0);
    for (int c = c0; c < c1; ++c) acc = cadd(acc, cmul(a[(size_t)c * n + row], x[(size_t)c * nrhs + r]));
    double* o = reinterpret_cast<double*>(Y + (size_t)b * n * nrhs + idx);
    atomicAdd(o, acc.x);
    atomicAdd(o + 1, acc.y);
}

cudaError_t matvec(int n, int batch, int nrhs, const double2* A, const double2* X, double2* Y, const int* active,
                   cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(Y, 0, sizeof(double2) * (size_t)batch * n * nrhs, s);
    if (e != cudaSuccess) return e;
    dim3 g((unsigned)(((size_t)n * nrhs + 255) / 256), (unsigned)((n + kMvCols - 1) / kMvCols), batch);
    matvec_kernel<<<g, 256, 0, s>>>(n, nrhs, A, X, Y, active);
    count_launch();
    return cudaGetLastError();
}

__global__ void c64_to_c128_kernel(int64_t count, const float2* s, double2* d) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < count; i += stride) d[i] = make_double2((double)s[i].x, (double)s[i].y);
}

// h[inst][i] (+)= <V_i, W> for i < k; inst = (b, r); grid (batch, nrhs)
__global__ void dots_kernel(int n, int nrhs, int k, const double2* V, size_t vstride, const double2* W,
                            double2* h, int hld, int accumulate, const int* active) {
    __shared__ double2 sh[kRed / 32];
    const int b = blockIdx.x, r = blockIdx.y;
    if (active && !active[b]) return;
    const size_t base = (size_t)b * n * nrhs + r;
    double2* hi = h + ((size_t)b * nrhs + r) * hld;
    for (int i = 0; i < k; ++i) {
        const double2* v = V + i * vstride + base;
        const double2* w = W + base;
        double2 acc = make_double2(0.0, 0.0);
        for (int row = threadIdx.x; row < n; row += kRed) acc = cadd(acc, cdotm(v[(size_t)row * nrhs], w[(size_t)row * nrhs]));
        double2 s = block_sum(acc, sh);
        if (threadIdx.x == 0) hi[i] = accumulate ? cadd(hi[i], s) : s;
    }
}

// nrm2[inst] = |W|^2
__global__ void norm2_kernel(int n, int nrhs, const double2* W, double* nrm2, const int* active) {
    __shared__ double2 sh[kRed / 32];
    const int b = blockIdx.x, r = blockIdx.y;
    if (active && !active[b]) return;
    const double2* w = W + (size_t)b * n * nrhs + r;
    double2 acc = make_double2(0.0, 0.0);
    for (int row = threadIdx.x; row < n; row += kRed) {
        const double2 v = w[(size_t)row * nrhs];
        acc.x += v.x * v.x + v.y * v.y;
    }
    double2 s = block_sum(acc, sh);
    if (threadIdx.x == 0) nrm2[(size_t)b * nrhs + r] = s.x;
}

// W -= sum_{i<k} h[inst][i] V_i
__global__ void update_kernel(int n, int nrhs, int batch, int k, const double2* V, size_t vstride, const double2* h,
                              int hld, double2* W, const int* active) {
    const size_t tot = (size_t)batch * n * nrhs;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int b = (int)(idx / ((size_t)n * nrhs)), r = (int)(idx % nrhs);
    if (active && !active[b]) return;
    const double2* hi = h + ((size_t)b * nrhs + r) * hld;
    double2 w = W[idx];
    for (int i = 0; i < k; ++i) {
        const double2 c = cmul(hi[i], V[i * vstride + idx]);
        w.x -= c.x;
        w.y -= c.y;
    }
    W[idx] = w;
}

// V = B - W
__global__ void sub_kernel(int n, int nrhs, int batch, const double2* B, const double2* W, double2* V,
                           const int* active) {
    const size_t tot = (size_t)batch * n * nrhs;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    if (active && !active[(int)(idx / ((size_t)n * nrhs))]) return;
    V[idx] = make_double2(B[idx].x - W[idx].x, B[idx].y - W[idx].y);
}

// V_out = W / sqrt(nrm2[inst]) (0 if the norm vanishes)
__global__ void scale_kernel(int n, int nrhs, int batch, const double2* W, const double* nrm2, double2* Vout,
                             const int* active) {
    const size_t tot = (size_t)batch * n * nrhs;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int b = (int)(idx / ((size_t)n * nrhs)), r = (int)(idx % nrhs);
    if (active && !active[b]) return;
    const double s2 = nrm2[(size_t)b * nrhs + r];
    const double f = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
    Vout[idx] = make_double2(W[idx].x * f, W[idx].y * f);
}

// Per instance: start a cycle (g = (beta, 0, ..)), or take column j of the
// Hessenberg matrix (h1 + h2, subdiagonal sqrt(nrm2)), apply the previous
// rotations, make the new one and update g; res = |g_{j+1}|.
struct Small {
    double2* H;      // [inst][m][m+1], column j at H + j (m+1)
    double2* g;      // [inst][m+1]
    double* c;       // [inst][m]
    double2* s;      // [inst][m]
    double* res;     // [inst]
    double2* y;      // [inst][m]
};

__global__ void cycle_start_kernel(int ninst, int nrhs, int m, const double* beta2, Small S, const int* active) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ninst || (active && !active[t / nrhs])) return;
    double2* g = S.g + (size_t)t * (m + 1);
    for (int i = 0; i <= m; ++i) g[i] = make_double2(0.0, 0.0);
    g[0] = make_double2(sqrt(beta2[t]), 0.0);
    S.res[t] = sqrt(beta2[t]);
}

__global__ void givens_kernel(int ninst, int nrhs, int m, int j, const double2* h1, const double2* h2,
                              const double* nrm2, Small S, const int* active) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ninst || (active && !active[t / nrhs])) return;
    double2* col = S.H + ((size_t)t * m + j) * (m + 1);
    for (int i = 0; i <= j; ++i) col[i] = cadd(h1[(size_t)t * (m + 1) + i], h2[(size_t)t * (m + 1) + i]);
    col[j + 1] = make_double2(sqrt(nrm2[t]), 0.0);
    double* c = S.c + (size_t)t * m;
    double2* s = S.s + (size_t)t * m;
    for (int i = 0; i < j; ++i) {
        const double2 a = col[i], b = col[i + 1];
        // [c s; -conj(s) c]
        const double2 sb = cmul(s[i], b);
        const double2 tmp = make_double2(c[i] * a.x + sb.x, c[i] * a.y + sb.y);
        const double2 csa = cmul(make_double2(s[i].x, -s[i].y), a);
        col[i + 1] = make_double2(c[i] * b.x - csa.x, c[i] * b.y - csa.y);
        col[i] = tmp;
    }
    const double2 a = col[j], b = col[j + 1];
    const double na = hypot(a.x, a.y), nb = hypot(b.x, b.y);
    double cj;
    double2 sj;
    if (na == 0.0) {
        cj = 0.0;
        sj = make_double2(1.0, 0.0);
        col[j] = b;
    } else {
        const double tt = hypot(na, nb);
        cj = na / tt;
        const double2 ph = make_double2(a.x / na, a.y / na);
        sj = cmul(ph, make_double2(b.x / tt, -b.y / tt));      // (a/|a|) conj(b)/t
        col[j] = make_double2(ph.x * tt, ph.y * tt);
    }
    col[j + 1] = make_double2(0.0, 0.0);
    c[j] = cj;
    s[j] = sj;
    double2* g = S.g + (size_t)t * (m + 1);
    const double2 gj = g[j];
    const double2 cg = cmul(make_double2(-sj.x, sj.y), gj);    // -conj(s) g_j
    g[j + 1] = cg;
    g[j] = make_double2(cj * gj.x, cj * gj.y);
    S.res[t] = hypot(cg.x, cg.y);
}

// y = H(0:k, 0:k)^{-1} g(0:k) per instance
__global__ void backsolve_kernel(int ninst, int nrhs, int m, int k, Small S, const int* active) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ninst || (active && !active[t / nrhs])) return;
    const double2* H = S.H + (size_t)t * m * (m + 1);
    const double2* g = S.g + (size_t)t * (m + 1);
    double2* y = S.y + (size_t)t * m;
    for (int i = k - 1; i >= 0; --i) {
        double2 v = g[i];
        for (int q = i + 1; q < k; ++q) {
            const double2 hy = cmul(H[(size_t)q * (m + 1) + i], y[q]);
            v.x -= hy.x;
            v.y -= hy.y;
        }
        const double2 d = H[(size_t)i * (m + 1) + i];
        const double dd = d.x * d.x + d.y * d.y;
        y[i] = dd > 0.0 ? make_double2((v.x * d.x + v.y * d.y) / dd, (v.y * d.x - v.x * d.y) / dd)
                        : make_double2(0.0, 0.0);
    }
}

// X += sum_{j<k} y_j Z_j
__global__ void xupdate_kernel(int n, int nrhs, int batch, int k, int m, const double2* Z, size_t vstride,
                               const double2* y, double2* X, const int* active) {
    const size_t tot = (size_t)batch * n * nrhs;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int b = (int)(idx / ((size_t)n * nrhs)), r = (int)(idx % nrhs);
    if (active && !active[b]) return;
    const double2* yi = y + ((size_t)b * nrhs + r) * m;
    double2 x = X[idx];
    for (int j = 0; j < k; ++j) x = cadd(x, cmul(yi[j], Z[j * vstride + idx]));
    X[idx] = x;
}

unsigned blocks_for(size_t tot) { return (unsigned)((tot + 255) / 256); }

}  // namespace

size_t gmres_scratch_bytes(int n, int batch, int nrhs, int m) {
    const size_t vec = (size_t)batch * n * nrhs * sizeof(double2), ninst = (size_t)batch * nrhs;
    return vec * (2 * (size_t)m + 2)                                    // V (m+1), Z (m), W
           + ninst * sizeof(double2) * ((size_t)m * (m + 1) + 3 * (m + 1) + 2 * (size_t)m)   // H, g, h1, h2, s, y
           + ninst * sizeof(double) * ((size_t)m + 4)                  // c, res, nrm2, beta2, |x|^2
           + (size_t)batch * n * nrhs * sizeof(float2)                 // FP32 solve buffer
           + 16 * 256;                                                 // alignment slack
}

int gmres_refine(int n, int batch, int nrhs, const double2* A, const float2* LU32, const int* piv,
                 const double2* B, double2* X, std::vector<int>& act, int* active_dev, void* scratch, int m,
                 int max_cycles, double tol, double tol_bw, double tol_floor, const std::vector<double>& an2,
                 cudaStream_t s, int& iters, std::vector<double>& mode_res, std::vector<double>& mode_bwd,
                 const float2* dinv, const int2* ptab) {
    const size_t vec = (size_t)batch * n * nrhs, ninst = (size_t)batch * nrhs;
    char* p = (char*)scratch;
    auto take = [&](size_t bytes) {
        char* q = p;
        p += (bytes + 255) & ~(size_t)255;
        return q;
    };
    double2* V = (double2*)take(vec * sizeof(double2) * (m + 1));
    double2* Z = (double2*)take(vec * sizeof(double2) * m);
    double2* W = (double2*)take(vec * sizeof(double2));
    Small S;
    S.H = (double2*)take(ninst * sizeof(double2) * m * (m + 1));
    S.g = (double2*)take(ninst * sizeof(double2) * (m + 1));
    double2* h1 = (double2*)take(ninst * sizeof(double2) * (m + 1));
    double2* h2 = (double2*)take(ninst * sizeof(double2) * (m + 1));
    S.s = (double2*)take(ninst * sizeof(double2) * m);
    S.y = (double2*)take(ninst * sizeof(double2) * m);
    S.c = (double*)take(ninst * sizeof(double) * m);
    S.res = (double*)take(ninst * sizeof(double));
    double* nrm2 = (double*)take(ninst * sizeof(double));
    double* beta2 = (double*)take(ninst * sizeof(double));
    double* xn2d = (double*)take(ninst * sizeof(double));
    float2* w32 = (float2*)take(vec * sizeof(float2));
    const dim3 gi(batch, nrhs);
    const unsigned ib = (unsigned)((ninst + 127) / 128);
    std::vector<double> res(ninst), bn2(ninst), rn2(ninst), xn2(ninst), target(ninst);
    std::vector<std::vector<double>> hist(ninst);
    cudaError_t e;
#define GM_TRY(x)                                                                                   \
    do {                                                                                            \
        if ((e = (x)) != cudaSuccess) return fail(PMLBIE_ECUDA, std::string("gmres: ") + cudaGetErrorString(e)); \
    } while (0)
    GM_TRY(cudaMemcpyAsync(active_dev, act.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s));
    // |B|^2 per instance
    norm2_kernel<<<gi, kRed, 0, s>>>(n, nrhs, B, nrm2, active_dev);
    count_launch();
    GM_TRY(cudaMemcpyAsync(bn2.data(), nrm2, sizeof(double) * ninst, cudaMemcpyDeviceToHost, s));
    iters = 0;
    for (int cyc = 0;; ++cyc) {
        // true residual r = B - A x -> V_0, beta^2 = |r|^2
        GM_TRY(matvec(n, batch, nrhs, A, X, W, active_dev, s));
        sub_kernel<<<blocks_for(vec), 256, 0, s>>>(n, nrhs, batch, B, W, V, active_dev);
        norm2_kernel<<<gi, kRed, 0, s>>>(n, nrhs, V, beta2, active_dev);
        norm2_kernel<<<gi, kRed, 0, s>>>(n, nrhs, X, xn2d, active_dev);
        count_launch(3);
        GM_TRY(cudaMemcpyAsync(rn2.data(), beta2, sizeof(double) * ninst, cudaMemcpyDeviceToHost, s));
        GM_TRY(cudaMemcpyAsync(xn2.data(), xn2d, sizeof(double) * ninst, cudaMemcpyDeviceToHost, s));
        GM_TRY(cudaStreamSynchronize(s));
        // converged: relative residual <= tol or normwise backward error
        // |r| / (|A|_F |x| + |b|) <= tol_bw, for every rhs of the mode
        int nact = 0;
        for (int b = 0; b < batch; ++b) {
            if (!act[b]) continue;
            double worst = 0.0, wbwd = 0.0;
            bool ok = true;
            for (int r = 0; r < nrhs; ++r) {
                const size_t t = (size_t)b * nrhs + r;
                const double rn = std::sqrt(rn2[t]), bn = std::sqrt(bn2[t]);
                const double den = std::sqrt(an2[b]) * std::sqrt(xn2[t]) + bn;
                const double rel = bn > 0 ? rn / bn : 0.0, bwd = den > 0 ? rn / den : 0.0;
                worst = std::max(worst, rel);
                wbwd = std::max(wbwd, bwd);
                if (!(rel <= tol || bwd <= tol_bw)) ok = false;
                target[t] = 0.5 * std::max(tol * bn, tol_bw * den);
                hist[t].clear();
            }
            // after a cycle: also done at the FP64 floor (backward error below
            // tol_floor that the last cycle did not halve)
            const bool floor = cyc > 0 && wbwd <= tol_floor && wbwd >= 0.5 * mode_bwd[b];
            mode_res[b] = worst;
            mode_bwd[b] = wbwd;
            if (ok || floor) act[b] = 0;
            else ++nact;
        }
        if (nact == 0 || cyc == max_cycles) break;
        GM_TRY(cudaMemcpyAsync(active_dev, act.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s));
        scale_kernel<<<blocks_for(vec), 256, 0, s>>>(n, nrhs, batch, V, beta2, V, active_dev);
        cycle_start_kernel<<<ib, 128, 0, s>>>((int)ninst, nrhs, m, beta2, S, active_dev);
        count_launch(2);
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double2* Vj = V + (size_t)j * vec;
            double2* Zj = Z + (size_t)j * vec;
            // z_j = (L U)^{-1} v_j: FP32 triangular solves (one CTA per system;
            // flexible GMRES absorbs their rounding)
            GM_TRY(convert_to_c64((int64_t)vec, Vj, w32, s));
            GM_TRY((batched_lu_solve<float2, float2>(n, batch, nrhs, LU32, piv, w32, s, active_dev, dinv, ptab)));
            c64_to_c128_kernel<<<(unsigned)std::min<size_t>(blocks_for(vec), 152 * 32), 256, 0, s>>>((int64_t)vec, w32, Zj);
            count_launch();
            GM_TRY(matvec(n, batch, nrhs, A, Zj, W, active_dev, s));
            dots_kernel<<<gi, kRed, 0, s>>>(n, nrhs, j + 1, V, vec, W, h1, m + 1, 0, active_dev);
            update_kernel<<<blocks_for(vec), 256, 0, s>>>(n, nrhs, batch, j + 1, V, vec, h1, m + 1, W, active_dev);
            dots_kernel<<<gi, kRed, 0, s>>>(n, nrhs, j + 1, V, vec, W, h2, m + 1, 0, active_dev);
            update_kernel<<<blocks_for(vec), 256, 0, s>>>(n, nrhs, batch, j + 1, V, vec, h2, m + 1, W, active_dev);
            norm2_kernel<<<gi, kRed, 0, s>>>(n, nrhs, W, nrm2, active_dev);
            givens_kernel<<<ib, 128, 0, s>>>((int)ninst, nrhs, m, j, h1, h2, nrm2, S, active_dev);
            scale_kernel<<<blocks_for(vec), 256, 0, s>>>(n, nrhs, batch, W, nrm2, V + (size_t)(j + 1) * vec, active_dev);
            count_launch(7);
            GM_TRY(cudaGetLastError());
            k = j + 1;
            ++iters;
            GM_TRY(cudaMemcpyAsync(res.data(), S.res, sizeof(double) * ninst, cudaMemcpyDeviceToHost, s));
            GM_TRY(cudaStreamSynchronize(s));
            // end the cycle when every instance met its target or stopped
            // improving (|g| not 20 % below its value four steps earlier)
            bool done = true;
            for (int b = 0; b < batch; ++b) {
                if (!act[b]) continue;
                for (int r = 0; r < nrhs; ++r) {
                    const size_t t = (size_t)b * nrhs + r;
                    hist[t].push_back(res[t]);
                    const size_t h = hist[t].size();
                    const bool stalled = h > 4 && res[t] > 0.8 * hist[t][h - 5];
                    if (res[t] > target[t] && !stalled) done = false;
                }
            }
            if (done) break;
        }
        backsolve_kernel<<<ib, 128, 0, s>>>((int)ninst, nrhs, m, k, S, active_dev);
        xupdate_kernel<<<blocks_for(vec), 256, 0, s>>>(n, nrhs, batch, k, m, Z, vec, S.y, X, active_dev);
        count_launch(2);
        GM_TRY(cudaGetLastError());
    }
#undef GM_TRY
    return PMLBIE_OK;
}

}  // namespace pmlbie
