// Internal declarations of the pmlbie library (host setup + CUDA kernels).
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pmlbie.h"

namespace pmlbie {

using cd = std::complex<double>;

constexpr int kStencil = 10;       // Lagrange stencil of the Alpert correction nodes
constexpr int kAlpertJ = 10;       // correction nodes per side (order-10 log rule)
constexpr int kAlpertA = 10;       // skipped grid neighbours per side

// Pair class of a grid node pair (l target, m source).
enum : uint8_t { kFar = 0, kNear = 1, kSkip = 2 };

// One close (or correction) pair: geometry the split kernels need, complex
// values stored as (re, im) doubles.  Layout shared by host and device.
struct NearPair {
    double2 d2;        // (rho~ - rho~')^2 + (z - z')^2
    double2 rr;        // rho~ rho~'
    double2 rho_t;     // target rho~
    double2 rho_s;     // source rho~'
    double2 drt;       // rho~' - rho~ (accurate for close points of a graded cluster)
    double2 nuc_r;     // source conormal (region a), rho component
    double2 nuc_z;     // source conormal (region a), z component
    double  dz;        // z - z' (target minus source, real on the curve)
    int     tgt;       // target unknown l
    int     src;       // grid-near: source unknown m; correction: correction index c
    int     flags;     // bit 0: correction pair; bit 1: far-by-criterion (plain FFT);
                       // bit 2: Taylor substitution (a point inside the PML)
    int     mirror = -1;   // grid-near: index of the pair with target and source
                           // exchanged (-1: none, or a correction pair)
};

enum { kFlagCorr = 1, kFlagFar = 2, kFlagSubst = 4 };

// Re(eta) M from which the close-pair Laplace modes take the downward
// (Miller) recurrence (below it, the upward one).
constexpr double kRecUpward = 3.5;
// Length of the recurrence tables: the downward recurrence starts at
// m_s = M + ceil(20 / Re(eta)) with Re(eta) M >= kRecUpward.
inline int rec_table_len(int M) { return M + (int)((20.0 * M) / kRecUpward) + 4; }

struct HostTables {
    int N = 0, Nt = 0, M = 0;
    double h = 0;
    std::vector<int> unk_grid;          // grid index of unknown l
    std::vector<int> unk_of_grid;       // inverse (-1 at breakpoints)
    // per unknown node
    std::vector<double> t, rho, z, speed, nu_r, nu_z, I, Wu, Wphi;
    std::vector<cd> rho_t, nuc_r, nuc_z;
    std::vector<int> bk;                 // nearest breakpoint of each node
    std::vector<double2> off;            // (rho, z) offset from it, accurate
    // Alpert rule
    std::vector<double> ax, aw;
    // correction points
    std::vector<int> corr_target;            // ncorr
    std::vector<double> corr_tau;            // ncorr
    std::vector<int> corr_m;                 // ncorr * kStencil (unknown or -1)
    std::vector<double> corr_coef;           // ncorr * kStencil (w_k h L)
    // correction points of target l: [corr_start[l], corr_start[l+1]); their
    // stencil columns lie in [corr_cmin[l], corr_cmin[l] + corr_w[l])
    std::vector<int> corr_start, corr_cmin, corr_w;
    int corr_wmax = 0;
    // classes and close pairs
    std::vector<uint8_t> cls;                // N*N, [l][m]
    std::vector<NearPair> near;              // grid-near pairs, then correction pairs
    int n_grid_near = 0;
    // pairs whose exact modal Laplace kernels are computed (one of a mirror
    // couple, none far by the criterion), grouped by arithmetic class and
    // recurrence length
    std::vector<int> near_lead;
    // diagonal
    std::vector<double> Da, Db;
};

struct DeviceTables {
    double *rho = nullptr, *z = nullptr, *I = nullptr, *Wu = nullptr, *Wphi = nullptr;
    double2 *rho_t = nullptr, *nuc_r = nullptr, *nuc_z = nullptr;
    int* bk = nullptr;
    double2* off = nullptr;
    uint8_t* cls = nullptr;
    NearPair* near = nullptr;
    int* near_lead = nullptr;
    int* corr_target = nullptr;
    int* corr_m = nullptr;
    double* corr_coef = nullptr;
    int* corr_start = nullptr;
    int* corr_cmin = nullptr;
    int* corr_w = nullptr;
    double *Da = nullptr, *Db = nullptr;
    double2* cos_tab = nullptr;   // (sin^2(psi_j/2), cos psi_j), j = 0..M/2
    double2* twid = nullptr;      // e^{-2 pi i e / M}, e = 0..M-1
    double2* twid2 = nullptr;     // e^{-2 pi i e / (2M)}, e = 0..2M-1
    // float-float copies for the mixed path's kernels (kernels_ff.cu): the
    // twiddles and angle table above as (re.hi, re.lo, im.hi, im.lo), the exp
    // and sin / cos tables of ffloat.cuh, and per node h W_u / (2M) and
    // h W_phi / (2M) (column weight times the trapezoid factor of the modes)
    // coefficients of the Legendre-Q three-term recurrence of the close-pair
    // Laplace modes, m = 0 .. kRecLen(M): upward (4m/(2m+1), (2m-1)/(2m+1)),
    // downward (4m/(2m-1), (2m+1)/(2m-1)) (entry 0 unused)
    double2* rec_up = nullptr;
    double2* rec_dn = nullptr;
    float4* twid_ff = nullptr;
    float4* twid2_ff = nullptr;
    float4* cos_ff = nullptr;
    float2* exp_ff = nullptr;
    float4* trig_ff = nullptr;
    float2* wuc_ff = nullptr;
    float2* wpc_ff = nullptr;
};

}  // namespace pmlbie

struct pmlbie_problem {
    pmlbie_params P;
    std::vector<double> vertices;
    double eta_split = 0;
    pmlbie::HostTables H;
    pmlbie::DeviceTables D;
    int device = 0;
    // workspace (allocated on first solve, grown as needed)
    void* ws = nullptr;
    size_t ws_bytes = 0;
    void* ws_extra = nullptr;   // device copies of per-node normals and speeds
    // far-pair counts for the report (computed once from H.cls): ordered far
    // pairs, those of two physical nodes, unordered pairs sampled, physical ones
    int far_counts[4] = {-1, -1, -1, -1};
};

namespace pmlbie {

// kernel launches issued by the library on this thread (read by the API calls)
extern thread_local long g_launches;
inline void count_launch(long n = 1) { g_launches += n; }

// errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
const char* error_text();
#define PMLBIE_CUDA_TRY(call)                                                    \
    do {                                                                         \
        cudaError_t _e = (call);                                                 \
        if (_e != cudaSuccess)                                                   \
            return ::pmlbie::fail(PMLBIE_ECUDA, std::string(#call) + ": " +      \
                                                    cudaGetErrorString(_e));     \
    } while (0)

// true once the problem's tables are on the device (api.cu)
bool device_ready(const pmlbie_problem* prob);

// host setup (host.cpp)
int build_tables(pmlbie_problem* prob);
void alpert_log_rule(int j, int a, std::vector<double>& x, std::vector<double>& w);

// kernels (kernels.cu)
struct FarLaunch {
    int mode_lo, mode_hi;
    // system-matrix output (column-major 2N x 2N per mode) or raw kernels
    double2* A;            // [mode][col][row], ld = 2N; may be null
    double2* raw;          // [mode][kernel][l][m]; may be null
    // the first launch for a (N, M, modes, output) shape may time the
    // candidate CTA sizes (it synchronises the stream once); false: never
    bool tune = false;
};
cudaError_t launch_far(const pmlbie_problem* prob, const FarLaunch& fl, cudaStream_t s);
// device time (ms) of the float-float far kernel's chosen configuration in its
// autotuning launch for this (N, M, modes, output) shape, run alone; 0 if not tuned
float far_ff_alone_ms(const pmlbie_problem* prob, int modes, bool raw);
// float-float far kernel of the mixed path (kernels_ff.cu); usable when
// far_ff_supported (every |q| of the problem inside its sin / cos range)
cudaError_t launch_far_ff(const pmlbie_problem* prob, const FarLaunch& fl, cudaStream_t s);
bool far_ff_supported(const pmlbie_problem* prob);
// host float-float tables of a problem with M azimuthal samples
void ff_tables(int M, std::vector<float4>& twid, std::vector<float4>& twid2, std::vector<float4>& cosv,
               std::vector<float2>& expv, std::vector<float4>& trig);
bool ff_elementary_known(int fn);
cudaError_t launch_ff_elementary(int fn, const double* x, double* out, size_t n, cudaStream_t s);
// pairs per CTA of this thread's last far-kernel launch (the tuned choice)
extern thread_local int g_far_pairs_per_cta;
// Per close pair, the float-float kernel's quantities (units of L = 2^eL):
// d~^2 / L^2, rho~ rho~' / L^2, the normal factor's two terms / L, omega_r L,
// 1 / (omega_r L), then eL and the all-real flag -- written by the Laplace-
// mode kernel (FP64, one pair per thread) into the float4 area that follows
// the Laplace modes in the zd scratch (kNearFF float4 per pair).
constexpr int kNearFF = 7;
// zd scratch of launch_near: Laplace modes [p][2][M], then, for ff, the
// per-pair float-float quantities
inline size_t near_zd_bytes(size_t np, int M, bool ff) {
    return sizeof(double2) * np * 2 * (size_t)M + (ff ? sizeof(float4) * kNearFF * np : 0);
}
// mid (optional): event recorded between the Laplace-mode and the modes kernels;
// ff: the modes kernel in float-float (mixed path; not with subst_off), zd
// sized by near_zd_bytes(.., true)
// mid_ff (optional): event recorded after the float-float modes kernel (right
// after mid when there is none)
cudaError_t launch_near(const pmlbie_problem* prob, int mode_lo, int mode_hi, double2* zd_scratch,
                        double2* out, cudaStream_t s, cudaEvent_t mid = nullptr, bool ff = false,
                        cudaEvent_t mid_ff = nullptr);
// the float-float close-pair modes kernel alone (kernels_ff.cu), after the
// Laplace modes are in zd
cudaError_t launch_near_modes_ff(const pmlbie_problem* prob, int mode_lo, int mode_hi, const double2* zd,
                                 const float4* pff, double2* out, cudaStream_t s);
// Taylor coefficients of cH1 (pa) and cH3 (pb) of degree L <= 7 (Sec. 4.3)
void taylor_coeffs(int L, double2* pa, double2* pb);
cudaError_t launch_near_to_raw(const pmlbie_problem* prob, int mode_lo, int mode_hi,
                               const double2* near_out, double2* raw, cudaStream_t s);
cudaError_t launch_assemble(const pmlbie_problem* prob, int mode_lo, int mode_hi,
                            const double2* near_out, double2* A, cudaStream_t s);
// rhs_par: per rhs kRhsPar doubles (sin phi, cos phi, R.re, R.im, k*.re, k*.im, azimuth, 0);
// nu_r, nu_z, speed per node; b1, b2 for modes [mode_lo, mode_hi)
constexpr int kRhsPar = 8;
// Raise a kernel's dynamic shared-memory limit to the device maximum minus its
// static shared memory.  Always the maximum, never the launch's own size:
// concurrent solves on several host threads set the same attribute, and a
// smaller value set by one would make another's larger launch fail.
template <typename K>
cudaError_t allow_max_smem(K kernel) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}
cudaError_t launch_rhs(const pmlbie_problem* prob, int n_rhs, int mode_lo, int mode_hi, const double* rhs_par_dev,
                       const double* nu_r, const double* nu_z, const double* speed, double2* b1, double2* b2,
                       cudaStream_t s);
// Point-source jumps (Sec. 2): per rhs, rhs_par holds rho_s, z_s at [0], [1] and
// the source azimuth at [6]; speed per node; b1, b2 for modes [mode_lo, mode_hi)
cudaError_t launch_point_rhs(const pmlbie_problem* prob, int n_rhs, int mode_lo, int mode_hi,
                             const double* rhs_par_dev, const double* speed, double2* b1, double2* b2,
                             cudaStream_t s);
// Waves (or sources) that share all but their azimuth: out[t][l][r] =
// e^{-i (mode_lo + t) az[r]} src[t][l][idx[r]] (src solved at azimuth 0 for the
// n_src distinct ones)
cudaError_t launch_expand_waves(int N, int nmodes, int mode_lo, int n_src, int n_rhs, const int* idx,
                                const double* az, const double2* src, double2* out, cudaStream_t s);
// Scattered-field modes at observation points (rho, z, region 0 upper / 1 lower,
// device arrays): coef scratch npts x N x (mode_hi - mode_lo) x 2 complex;
// densities and out laid out [mode - mode_lo][node or point][rhs]
cudaError_t launch_field(const pmlbie_problem* prob, int npts, const double* prho, const double* pz,
                         const int* preg, int mode_lo, int mode_hi, int nrhs, const double2* u1,
                         const double2* phi1, const double2* u2, const double2* phi2, double2* coef, double2* out,
                         cudaStream_t s);
// nm: modes in the chunk (A, b1, b2, B, X hold nm modes)
cudaError_t launch_block_rhs(const pmlbie_problem* prob, int n_rhs, int nm, const double2* A,
                             const double2* b1, const double2* b2, double2* B, cudaStream_t s);
cudaError_t launch_outputs(const pmlbie_problem* prob, int n_rhs, int nm, const double2* X,
                           const double2* b1, const double2* b2, double2* u1, double2* phi1,
                           double2* u2, double2* phi2, cudaStream_t s);

// Elementary-function self-test (pmlbie_selftest_elementary): the functions
// selected by fn at n points, out as documented in include/pmlbie.h
bool elementary_selftest_known(int fn);
cudaError_t launch_elementary_selftest(int fn, const double* x, double* out, size_t n, cudaStream_t s);

// Pipe-throughput probes (probe.cu): kind 0 FP64 FMA, 1 FP32 FMA, 2 TF32
// tcgen05 MMA; TFLOP/s of one timed launch over every SM
int peak_probe(int kind, double* out_tflops, cudaStream_t s);

// dense batched linear algebra (lu.cu)
// Leaves piv[b] as the row permutation of the factorisation: piv[b][i] is the
// original row that ends in row i (P A = L U with (P x)_i = x_{piv[i]}).
// upd_ev: optional 2 x ceil(n/32) events recorded around each trailing update
// (its update launch, with its operand-image launch when that is on s; for its
// timing; recorded as external events, so that they become event-record nodes
// when the factorisation is captured in a graph)
// img: for complex64, lu_image_bytes(n, batch) bytes of device scratch (16-byte
// aligned) holding one step's split operand images; unused for complex128
// ptab: for complex64, lu_ptab_elems(n, batch) entries receiving each step's
// row-interchange mapping: the interchanges are applied to the columns right of
// each panel only (L keeps the row order of its step), piv keeps LAPACK's
// interchange indices, and the solves take ptab; unused for complex128 (L in
// getrf's row order, piv the row permutation)
// side: for complex64, an auxiliary stream and two events (created outside any
// capture); each step's A' images (which need only the panel) then run on it
// beside the row-swap / block-row-solve kernel; null: all on s
struct LuSide {
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
template <typename T>
cudaError_t batched_lu(int n, int batch, T* A, int* piv, int* info, cudaStream_t s, unsigned char* img,
                       int2* ptab, const LuSide* side = nullptr, cudaEvent_t* upd_ev = nullptr);
size_t lu_ptab_elems(int n, int batch);
// scratch bytes of the complex64 factorisation's operand images (the first
// step's 64-row blocks of L21 and 64-column blocks of U12, 96 KB per pair)
size_t lu_image_bytes(int n, int batch);
// kernel attributes of batched_lu<T>, set once (call before capturing it)
template <typename T>
cudaError_t lu_prepare();
// active: optional per-matrix flags (0 = skip), used to leave converged modes alone
// factors in TF, right-hand sides and arithmetic in T (T = double2 with TF = float2:
// FP64 solves with the FP32 factors)
// dinv: optional inverses of the 32 x 32 diagonal blocks (batched_diag_inv),
// used when n is a multiple of 32
template <typename T, typename TF>
// ptab: the complex64 factorisation's interchange mapping (batched_lu); then
// piv is not read
cudaError_t batched_lu_solve(int n, int batch, int nrhs, const TF* LU, const int* piv, T* B,
                             cudaStream_t s, const int* active = nullptr, const TF* dinv = nullptr,
                             const int2* ptab = nullptr);
// inverses of the 32 x 32 diagonal blocks of L (unit lower) and U of every
// complex64 factor, [b][n / 32][2][32 x 32] column-major (n a multiple of 32)
cudaError_t batched_diag_inv(int n, int batch, const float2* LU, float2* dinv, cudaStream_t s);
inline size_t diag_inv_elems(int n) { return (size_t)n * 64; }   // per matrix
cudaError_t convert_to_c64(int64_t count, const double2* src, float2* dst, cudaStream_t s);
// complex64 copies of batch n x n complex128 matrices and their squared
// Frobenius norms (out[b] = |A_b|_F^2) in one pass over A
cudaError_t convert_fro2_c128(int n, int batch, const double2* A, float2* A32, double* out, cudaStream_t s);
// Flexible GMRES (FP64, right-preconditioned by the FP32 LU) for the modes with
// act[b] = 1; X holds the start and receives the solution; act is cleared for
// converged modes (relative residual <= tol or normwise backward error
// |r| / (|A|_F |x| + |b|) <= tol_bw; an2 = |A_b|_F^2), mode_res / mode_bwd
// receive their final relative residuals and backward errors.
size_t gmres_scratch_bytes(int n, int batch, int nrhs, int m);
int gmres_refine(int n, int batch, int nrhs, const double2* A, const float2* LU32, const int* piv,
                 const double2* B, double2* X, std::vector<int>& act, int* active_dev, void* scratch, int m,
                 int max_cycles, double tol, double tol_bw, double tol_floor, const std::vector<double>& an2,
                 cudaStream_t s, int& iters, std::vector<double>& mode_res, std::vector<double>& mode_bwd,
                 const float2* dinv = nullptr, const int2* ptab = nullptr);
// R = B - A X with |R|^2, |B|^2, |X|^2 per (matrix, rhs)
cudaError_t residual_c128(int n, int batch, int nrhs, const double2* A, const double2* X,
                          const double2* B, double2* R, double* rnorm, double* bnorm, double* xnorm,
                          cudaStream_t s, const int* active = nullptr);
cudaError_t refine_step(int n, int batch, int nrhs, const float2* LU32, const int* piv,
                        const double2* R, float2* work32, double2* X, cudaStream_t s,
                        const int* active = nullptr, const float2* dinv = nullptr, const int2* ptab = nullptr);

}  // namespace pmlbie
