/*
 * pmlbie.h - C ABI of the GB300 (sm_103a) PML-BIE modal solver.
 *
 * The library solves 3D acoustic transmission through a two-layer medium whose
 * interface is the plane z = 0 with an axisymmetric perturbation, truncated by a
 * cylindrical PML, with the Fourier-mode boundary integral method of Wang & Lu,
 * "An FFT-accelerated PML-BIE solver for three-dimensional acoustic wave
 * scattering in layered media" (arXiv 2412.11162):
 *
 *   Sec. 2    problem statement: wavenumbers omega_1 (z above the interface) and
 *             omega_2 (below), plane-wave incidence, reference field u^{tot,0}.
 *   Sec. 3.1  PML stretching rho~ = rho + i int sigma_1 (Eq. (sgm1)) and the
 *             PML Green's function with a complex distance.
 *   Sec. 3.3  azimuthal Fourier modes; decoupled modal equations (Eq. (6)).
 *   Sec. 4.1  graded mesh (Eq. (sxi)), kernel splitting (Eqs. (s1), (k1)),
 *             FFT modal kernels, Alpert quadrature, NtD matrices.
 *   Sec. 4.2  transmission coupling of the two regions, right-hand sides b^1, b^2.
 *   Sec. 4.3  stabilised distance and the cH_1 / cH_3 substitution.
 *
 * Conventions
 *   - Every call returns an int status: PMLBIE_OK (0) or a negative error code.
 *     pmlbie_last_error() returns a message owned by the library (per thread).
 *   - Device pointers are CUDA global-memory addresses on the current device;
 *     host pointers are ordinary CPU memory.  "stream" is a cudaStream_t passed
 *     as void* (NULL = legacy default stream).  All device work is ordered on
 *     that stream; host-buffer calls synchronise it before returning.
 *   - Complex numbers are interleaved (re, im) doubles (complex128) unless a
 *     call says otherwise.
 *   - Modes: the modal kernels are F^_n = int_{-pi}^{pi} e^{-i n psi} F dpsi.
 *     All kernels are even in psi, so F^_{-n} = F^_n; the library computes the
 *     distinct modes n = 0 .. M/2-1 (Sec. 3.3).
 *   - Unknowns: N nodes on the generating curve gamma_AB (axis point A to the
 *     PML end B = (a1 + T, 0)); breakpoints of the graded grid carry none.
 */
#ifndef PMLBIE_H
#define PMLBIE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PMLBIE_OK            0
#define PMLBIE_EINVAL      (-1)   /* invalid parameter or size                    */
#define PMLBIE_ENOMEM      (-2)   /* device or host allocation failed             */
#define PMLBIE_ECUDA       (-3)   /* a CUDA call failed                           */
#define PMLBIE_ESINGULAR   (-4)   /* zero pivot in a modal LU factorisation       */
#define PMLBIE_ENOCONVERGE (-5)   /* iterative refinement missed its tolerance    */
#define PMLBIE_ENAN        (-6)   /* NaN or Inf in an output                      */
#define PMLBIE_ENODEV      (-7)   /* no CUDA device / extension not usable        */
#define PMLBIE_ETIMEOUT    (-8)   /* a device-side bounded wait expired           */

/* generating-curve kinds */
#define PMLBIE_CURVE_GAUSS_BUMP 0   /* z = h (e^{-r^2/w} - e^{-R^2/w})/(1 - e^{-R^2/w}), r <= R; flat to B */
#define PMLBIE_CURVE_POLYLINE   1   /* vertices (rho, z) from the axis; flat to B appended if needed     */
#define PMLBIE_CURVE_WAVY_DENT  2   /* Sec. 5 Example 2: rho = f sin(pi s/2), z = -f cos(pi s/2),
                                       f = R (1 - eps sin(m pi s)), s in [0, 1]; flat to B            */

/* arithmetic of a solve */
#define PMLBIE_FP64  0   /* everything in FP64 (complex128)                          */
#define PMLBIE_MIXED 1   /* FP64 modal kernels, FP32 LU, FP64 iterative refinement    */

/* Problem statement (Sec. 2, Sec. 3.1, Sec. 4, Sec. 5).  Owned by the caller;
 * pmlbie_create copies what it needs. */
typedef struct {
    uint32_t struct_size;     /* sizeof(pmlbie_params)                                */
    double   k1, k2;          /* omega_1 (upper medium), omega_2 (lower medium) > 0  */
    double   a1, T, S;        /* PML start radius, thickness, strength (Eq. (sgm1))  */
    int      p;               /* PML profile and grading exponent (Sec. 5: 6), >= 2  */
    int      N;               /* unknown nodes on gamma_AB, >= 32                    */
    int      M;               /* azimuthal samples, 2^a 3^b, 4 | M, 16 <= M <= 768   */
    int      curve_kind;      /* PMLBIE_CURVE_*                                       */
    double   bump_h, bump_w, bump_R;   /* Gaussian bump (kind 0)                     */
    int      n_vertices;      /* polyline (kind 1): vertex count                     */
    const double* vertices;   /* polyline: n_vertices (rho, z) pairs, host memory    */
    int      taylor_L;        /* degree of the cH_1 / cH_3 substitution (Sec. 4.3: 5) */
    double   split_c;         /* close-pair threshold eta_s = split_c * 2 pi / M      */
    double   wavy_R, wavy_eps;  /* wavy dent (kind 2): 0 < R <= a1, 0 <= eps < 1        */
    int      wavy_m;            /* wavy dent: half-waves, 1..64 (Example 2: 1, 0.1, 3)  */
    int      subst_off;         /* diagnostic: 1 = exact split (H1 = cos q, H3 = cos q +
                                   q sin q) on close pairs with a PML point too, the
                                   "without cH1" arm of Sec. 4.3 (unstable for strong
                                   PMLs); 0 = the cH1 / cH3 substitution (default)      */
} pmlbie_params;

/* Report of a solve (filled when the pointer is not NULL). */
typedef struct {
    uint32_t struct_size;
    int      n_modes;             /* M/2                                              */
    int      near_pairs;          /* close pairs evaluated with the kernel split       */
    int      refine_iters;        /* max refinement iterations over modes (mixed)      */
    double   residual;            /* max over modes/RHS of ||B - A x|| / ||B||         */
    double   ms_kernels;          /* device time: modal kernels + assembly, + rhs in the FP64
                                     path (the mixed path forms the right-hand sides beside
                                     its factorisation) (ms)                                */
    double   ms_lu;               /* device time: factorisation (mixed: complex64 conversion,
                                     LU and diagonal-block inverses, on a high-priority stream
                                     beside the right-hand sides) (ms)                      */
    double   ms_solve;            /* device time: solves + refinement + outputs (ms)   */
    double   ms_far;              /* device time of the far-pair kernel launch (ms); it
                                     runs beside the close-pair kernels, so ms_far and
                                     ms_near overlap                                      */
    double   ms_near;             /* device time of the close-pair kernels, on their own
                                     high-priority stream (ms)                            */
    double   ms_assemble;         /* device time of Alpert assembly + diagonal (ms)    */
    int      launches;            /* CUDA kernel launches issued by the call           */
    int      far_pairs;           /* node pairs evaluated by the far-pair FFT kernel   */
    double   ms_near_laplace;     /* device time of the close-pair Laplace-mode kernel
                                     (part of ms_near) (ms)                            */
    int      chunks;              /* mode chunks the solve was split into              */
    int      chunk_modes;         /* modes per chunk                                   */
    int      gmres_modes;         /* mixed: modes finished by FGMRES (refinement stalled) */
    int      gmres_iters;         /* mixed: FGMRES iterations (max over chunks)        */
    double   backward_error;      /* mixed: max over modes/RHS of |B - A x| / (|A|_F |x| + |B|) */
    int      far_pairs_physical;  /* far pairs with both nodes outside the PML (real distance) */
    int      lu_graph_replays;    /* LU factorisations replayed from a captured CUDA graph */
    int      far_pairs_per_cta;   /* node pairs per CTA of the far-pair kernel (autotuned) */
    int      far_pairs_sampled;   /* unordered pairs {l, m} sampled by the far-pair kernel: one
                                     sampling and one set of transforms serves both (l, m) and
                                     (m, l) (S~ is symmetric, K~ differs by its normal factor) */
    int      far_pairs_sampled_physical;  /* of those, pairs of two physical nodes           */
    double   ms_near_ff;          /* mixed: device time of the float-float close-pair modes kernel
                                     (pairs without a PML point; part of ms_near) (ms) */
    double   ms_lu_update;        /* device time of the LU's trailing updates, summed (part of
                                     ms_lu; an event pair around each step's operand-image and
                                     tensor-core update launches) (ms) */
    int      lu_update_launches;  /* trailing updates (steps with a trailing matrix) of those
                                     factorisations, each timed by one event pair             */
    double   ms_far_alone;        /* mixed: device time of the float-float far-pair kernel run
                                     alone (its autotuning launch of the chosen CTA size, on the
                                     first solve of this shape; 0 when not tuned) (ms)          */
} pmlbie_report;

/* Options of pmlbie_solve_ex (zero-initialise, then set struct_size). */
typedef struct {
    uint32_t struct_size;         /* sizeof(pmlbie_solve_opts)                                  */
    int      precision;           /* PMLBIE_FP64 or PMLBIE_MIXED                                */
    int      n_rhs;               /* plane waves, 1..4096                                        */
    const double* polar;          /* host, n_rhs polar angles in [0, pi/2) (from the z axis)    */
    const double* azimuth;        /* host, n_rhs incidence azimuths (NULL: all 0)               */
    int      mode_lo, mode_hi;    /* modes solved, [mode_lo, mode_hi) in [0, M/2); 0, 0 = all   */
    int      max_chunk_modes;     /* modes per chunk at most (0: no cap)                        */
    size_t   workspace_limit;     /* device workspace bytes at most (0: 90 % of free memory)    */
    const double* source_rho;     /* host, n_rhs point sources instead of plane waves (with    */
    const double* source_z;       /* polar = NULL): source r at (source_rho[r], azimuth[r],     */
                                  /* source_z[r]) in the upper medium (NULL: plane waves)       */
} pmlbie_solve_opts;

typedef struct pmlbie_problem pmlbie_problem;   /* opaque, owned by the library */

/* Build the geometry, PML tables, Alpert quadrature, close-pair lists and the
 * diagonal term on the host.  Nothing touches a GPU here: the tables are
 * uploaded to the then-current CUDA device by the first device call
 * (pmlbie_modal_kernels / pmlbie_solve*), which must run on that device from
 * then on.  Errors: EINVAL (parameter check), ENOMEM. */
int  pmlbie_create(const pmlbie_params* params, pmlbie_problem** out);

/* Release every host and device resource of the problem (NULL is ignored). */
void pmlbie_destroy(pmlbie_problem* prob);

/* Message for the last error raised on the calling thread (never NULL). */
const char* pmlbie_last_error(void);

/* Node tables (host copies, length N each, any pointer may be NULL):
 * rho, z of the nodes, |r'(t)| and the curve parameter t.  EINVAL if n != N. */
int  pmlbie_nodes(const pmlbie_problem* prob, double* rho, double* z, double* speed,
                  double* t, int n);

/* Diagonal term D (Sec. 3.2 Lemmas 3.1-3.3, Sec. 4.1) of both regions, host
 * copies of length N.  D^a uses the outward normal of the upper region, D^b
 * that of the lower region. */
int  pmlbie_diagonal(const pmlbie_problem* prob, double* Da, double* Db, int n);

/* Sizes of the problem: N unknown nodes and M azimuthal samples (modes
 * 0 .. M/2-1), as given to pmlbie_create (Sec. 3.3, Sec. 4.1).  Either
 * pointer may be NULL.  EINVAL if prob is NULL. */
int  pmlbie_dims(const pmlbie_problem* prob, int* N, int* M);

/* Number of close (split) pairs: grid pairs and Alpert correction pairs. */
int  pmlbie_near_count(const pmlbie_problem* prob, int* n_grid_near, int* n_corr);

/* Host copy of the close-pair list (Sec. 4.1 kernel splitting; the pairs with
 * Re sqrt(d~^2 / (rho~ rho~')) below the split threshold, plus every Alpert
 * correction pair), n = n_grid_near + n_corr entries in the library's order:
 * the grid pairs by target, then source; then the correction pairs in the
 * order of their correction points (target, side, node of the rule).  Per
 * entry: tgt (unknown l), src (grid: unknown m; correction: the correction
 * point's index), flags (bit 0: correction pair; bit 1: a correction pair
 * that is far by the criterion and takes the plain FFT; bit 2: Taylor
 * substitution of Sec. 4.3, a point inside the PML), mirror (grid pairs:
 * index of the pair with target and source exchanged, -1 if that pair is not
 * close; correction pairs: -1).  Any pointer may be NULL.  EINVAL if n is not
 * the list's length. */
int  pmlbie_near_pairs(const pmlbie_problem* prob, int* tgt, int* src, int* flags, int* mirror, int n);

/* Host copy of the Alpert correction table (Sec. 4.1 Eqs. (snab1), (snt1)):
 * n = n_corr correction points (pmlbie_near_count) in the order of the
 * close-pair list's correction pairs.  Per point c: target[c] (unknown l),
 * tau[c] (curve parameter of the point, in (0, 1)), and the PMLBIE_STENCIL
 * unknowns m[c * PMLBIE_STENCIL + a] (-1 at breakpoints) of its Lagrange
 * stencil with coefficients coef[...] = w_k h L_a(tau) (Alpert weight times
 * grid step times Lagrange weight); the correction adds coef x W(m) x F(r_l,
 * r(tau)) to column m.  Any pointer may be NULL.  EINVAL if n is not n_corr. */
#define PMLBIE_STENCIL 10

/* Host copy of the per-node PML and quadrature tables (length N each, any
 * pointer may be NULL): I = int_{a1}^{rho} sigma (Sec. 3.1 Eq. (rhot), so the
 * stretched radius is rho~ = rho + i I), the conormal nu_c of region a as
 * complex pairs (re, im) interleaved: nuc_r[2 l], nuc_r[2 l + 1] (Sec. 3.1,
 * nu_c = (nu_rho rho~ alpha_z / (rho alpha_rho), nu_z rho~ alpha_rho / (rho
 * alpha_z)) with alpha = 1 + i sigma), and the column weights Wu = 2 rho |r'|
 * (double-layer / u columns) and Wphi = 2 rho (single-layer / phi columns)
 * of the graded trapezoid.  EINVAL if n != N. */
int  pmlbie_node_tables(const pmlbie_problem* prob, double* I, double* nuc_r, double* nuc_z, double* Wu,
                        double* Wphi, int n);
int  pmlbie_corrections(const pmlbie_problem* prob, int* target, double* tau, int* m, double* coef, int n);

/* Alpert's log-singular end correction used by the quadrature (Sec. 4.1,
 * order 10 in Sec. 5): j nodes x[k] in (0, a) and weights w[k] (host arrays of
 * length j), generated by the library from the rule's moment conditions.
 * Supported: 2 <= j <= 12, 1 <= a <= 16.  EINVAL otherwise or if the solve
 * for the rule fails. */
int  pmlbie_alpert_rule(int j, int a, double* x, double* w);

/* Bytes of device workspace a solve of all modes with n_rhs right-hand sides
 * allocates (kept by the problem for the next solve).  A mixed solve whose
 * refinement hands modes to FGMRES allocates its Krylov bases (42 vectors of
 * the chunk's right-hand sides) for the duration of that step only. */
size_t pmlbie_workspace_bytes(const pmlbie_problem* prob, int precision, int n_rhs);

/* Modal kernels S^_n, K^_n of both regions on every grid node pair (Sec. 4.1,
 * Eqs. (snspml), (knspml)): far pairs by the M-point FFT in psi, close pairs
 * by the kernel split, pairs inside the Alpert skip band (|i - j| < 10 grid
 * steps) set to 0.  Output: dev_out, caller-owned device buffer of
 * (mode_hi - mode_lo) * 4 * N * N complex128 laid out
 * [mode][kernel][l][m], kernel = 0: S^a, 1: K^a, 2: S^b, 3: K^b (region a =
 * upper medium with omega_1 and normal nu; region b = lower medium, omega_2,
 * normal -nu), l = target node, m = source node.  0 <= mode_lo < mode_hi <= M/2. */
int  pmlbie_modal_kernels(pmlbie_problem* prob, int mode_lo, int mode_hi, void* dev_out,
                          void* stream);

/* pmlbie_modal_kernels in the arithmetic of a solve's precision: PMLBIE_FP64
 * as pmlbie_modal_kernels; PMLBIE_MIXED as the mixed solve builds its
 * matrices: the far pairs' samples, transforms and scatter, and the close
 * pairs' split samples, transforms and convolution, in float-float (pairs
 * of FP32 numbers, ~48-bit significands, on the FP32 pipe; relative rounding
 * ~1e-14 of a pair's samples, growing with |q| = omega |dr| as |q| 2^-47),
 * with the exact modal Laplace kernels of the split (Sec. 4.1, the
 * near-singular part) in FP64.  Problems whose phases |q| reach the
 * float-float sin / cos range (~780), and the diagnostic exact split
 * (subst_off), take the FP64 kernels in both precisions.
 * Errors as pmlbie_modal_kernels; EINVAL for another precision. */
int  pmlbie_modal_kernels_ex(pmlbie_problem* prob, int precision, int mode_lo, int mode_hi, void* dev_out,
                             void* stream);

/* Split modal kernels of every close pair (Sec. 4.1 kernel splitting; Sec. 4.3
 * substitution on PML pairs), in the close-pair list's order (pmlbie_near_pairs:
 * grid pairs, then Alpert correction pairs -- the values the assembly adds
 * with the Lagrange stencils), in the arithmetic of `precision` as
 * pmlbie_modal_kernels_ex.  Output: dev_out, caller-owned device buffer of
 * (n_grid_near + n_corr) * 4 * (mode_hi - mode_lo) complex128 laid out
 * [pair][kernel][mode], kernel as in pmlbie_modal_kernels; no quadrature
 * weights.  Synchronises the stream.  Errors as pmlbie_modal_kernels_ex. */
int  pmlbie_close_pair_kernels(pmlbie_problem* prob, int precision, int mode_lo, int mode_hi, void* dev_out,
                               void* stream);

/* Allocation-free variant of pmlbie_modal_kernels (the paper has no
 * counterpart: this is a deployment convenience).  For callers that must not
 * call cudaMalloc while they run (a framework whose own allocator owns the
 * device memory budget, or an embedding that forbids driver allocations
 * after start-up).  Same output, layout and arguments as
 * pmlbie_modal_kernels; the close-pair scratch lives in one file-scope device
 * array of 64 MiB per device (held by every device that loads the library
 * until the process exits) instead of being allocated.
 *   - The problem's tables must already be on the current device (a prior
 *     pmlbie_modal_kernels or pmlbie_solve on it); otherwise EINVAL.
 *   - Problems whose close-pair scratch, N_close * (2 M + 4 (mode_hi -
 *     mode_lo)) * 16 bytes, exceeds 64 MiB are rejected with EINVAL (ask
 *     for fewer modes per call, or use pmlbie_modal_kernels).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call shares the array: calls whose work overlaps on the GPU (for
 *     instance on two streams) race; order them on one stream.  Nothing in
 *     the array needs to start at zero.
 *   - The call is stream-ordered and does not synchronise: dev_out is ready
 *     when the stream reaches the end of the call's work. */
int  pmlbie_modal_kernels_noalloc(pmlbie_problem* prob, int mode_lo, int mode_hi, void* dev_out,
                                  void* stream);

/* Full solve for plane waves of polar angles polar[0..n_rhs-1] (azimuth 0),
 * Sec. 4.1-4.2: kernels, split, Alpert assembly, diagonal, right-hand side,
 * batched LU per mode, solves (and FP64 refinement for PMLBIE_MIXED).
 * Outputs (caller-owned device buffers, complex128, [mode][node][rhs], M/2
 * modes): u1 = u^{s,1}_n, phi1 = |r'| d_nu_c u^{s,1}_n, u2, phi2 (the same for
 * the lower medium, d_nu with the same nu).  Any output may be NULL.
 * Mixed precision: modal kernels in float-float arithmetic on the FP32 pipe
 * (as pmlbie_modal_kernels_ex with PMLBIE_MIXED) stored as complex128
 * matrices, complex64 LU (tensor-core trailing updates), iterative
 * refinement with FP64 residuals of those matrices until, for
 * every mode and right-hand side, the relative residual is <= 1e-13, or the
 * normwise backward error |B - A x| / (|A|_F |x| + |B|) is <= 1e-16, or it is
 * <= 1e-14 and no longer decreasing (the FP64 floor); modes
 * whose refinement stalls (condition number x FP32 LU error near 1 or above)
 * are restarted and solved by flexible GMRES in FP64 preconditioned by the
 * same LU.  Errors: EINVAL, ENOMEM, ECUDA, ESINGULAR, ENOCONVERGE (mixed: a
 * mode missed both tolerances after the iteration caps; outputs still
 * written), ETIMEOUT (a bounded wait of the tensor-core LU update expired),
 * ENAN (NaN or Inf in an output; outputs written).  Inside the call some
 * kernels run on the problem's own streams (the close-pair kernels beside
 * the far-pair kernel; in the mixed path the factorisation beside the
 * right-hand sides), forked from `stream` after the work already queued on
 * it and joined back into it; one problem serves one call at a time. */
int  pmlbie_solve(pmlbie_problem* prob, int precision, int n_rhs, const double* polar,
                  void* dev_u1, void* dev_phi1, void* dev_u2, void* dev_phi2,
                  void* stream, pmlbie_report* rep);

/* Solve with options (Sec. 4.1-4.2 as pmlbie_solve): incidence azimuths, a
 * mode range, and mode chunking.  Modes are independent (Sec. 3.3), so the
 * call processes [mode_lo, mode_hi) in chunks of at most max_chunk_modes modes
 * whose workspace fits workspace_limit: each chunk samples the kernels, builds
 * and factors its systems and solves them before the next starts (the kernel
 * sampling is repeated per chunk).  Plane wave r has polar angle polar[r] and
 * azimuth azimuth[r]; mode n of its data is e^{-i n azimuth} times that of the
 * azimuth-0 wave (modes -n follow as e^{+i n azimuth} times the same); waves
 * that share a polar angle are therefore solved once, at azimuth 0, and
 * rotated into their outputs (the call then holds device buffers for the
 * distinct angles' solutions for its duration).
 * Point sources (Sec. 2, spherical incidence; source_rho, source_z set and
 * polar NULL): the incident field of source r is G_1(x, x_s) with x_s =
 * (source_rho[r], azimuth[r], source_z[r]) in the upper medium; the jumps are
 * b^1 = -G~_1(r~, x_s), b^2 = -|r'| d_nu_c G~_1 at every node (PML nodes in
 * stretched coordinates), their modes the M-point DFTs in psi (the far-pair
 * rule).  u1, phi1 then hold the scattered field above and u2, phi2 the total
 * field below.  Each source needs 0 <= rho_s < a1, z_s finite, and every node
 * at a separation d / sqrt(rho_s rho_m) >= split_c * 2 pi / M (the far-pair
 * criterion, so that the M-point rule resolves the data); the caller places
 * it above the interface.  Sources that share (rho_s, z_s) are solved once
 * and rotated, as plane waves that share a polar angle.
 * Outputs as pmlbie_solve with (mode_hi - mode_lo) modes:
 * [mode - mode_lo][node][rhs].  Synchronises the stream at the end of every
 * chunk.  Errors as pmlbie_solve; ENOMEM if one mode does not fit the limit. */
int  pmlbie_solve_ex(pmlbie_problem* prob, const pmlbie_solve_opts* opts, void* dev_u1, void* dev_phi1,
                     void* dev_u2, void* dev_phi2, void* stream, pmlbie_report* rep);

/* Several independent problem instances (different wavenumbers, geometries,
 * sizes, right-hand sides), each solved as pmlbie_solve_ex with opts[i] into
 * dev_u1[i] .. dev_phi2[i] (any of the four arrays may be NULL, and any entry
 * NULL).  Instances are spread over n_streams (1..8) internal streams, each
 * driven by its own host thread, so that the latency-bound phases of one
 * instance (panel factorisation, refinement checks) overlap the work of
 * another; the internal streams start after the work already queued on
 * `stream`, and `stream` waits for all of them.  release_workspace != 0 frees
 * each instance's device workspace after its solve (peak memory = n_streams
 * workspaces).  reps: n_probs reports or NULL.  The problems must be
 * distinct.  Returns the first failing instance's status (all instances are
 * attempted). */
int  pmlbie_solve_batch(pmlbie_problem* const* probs, int n_probs, const pmlbie_solve_opts* opts,
                        void* const* dev_u1, void* const* dev_phi1, void* const* dev_u2, void* const* dev_phi2,
                        int n_streams, int release_workspace, void* stream, pmlbie_report* reps);

/* Scattered field at observation points (Sec. 4.2, Eq. (fujs)): the modal
 * representation formula of each medium with the solved densities,
 *   upper medium:  u^{s,1}_n(x) =  1/2 sum_m h [W_phi S^a_n(x, r_m) phi1_m - W_u K^a_n(x, r_m) u1_m]
 *   lower medium:  u^{s,2}_n(x) = -1/2 sum_m h [W_phi S^b_n(x, r_m) phi2_m + W_u K^b_n(x, r_m) u2_m]
 * (W_u = 2 rho |r'|, W_phi = 2 rho, K^b with the normal -nu; the modal kernels
 * by the M-point rule in psi).  Points: host arrays rho[p], z[p] with
 * 0 <= rho < a1 (physical region) and region[p] = 0 (upper, omega_1) or 1
 * (lower, omega_2); they must lie well off the curve (several node spacings:
 * no near-field correction is applied).  Densities: device buffers as written
 * by pmlbie_solve_ex for modes [mode_lo, mode_hi) and n_rhs waves,
 * [mode - mode_lo][node][rhs] (those of a medium without points may be NULL);
 * mode_lo = mode_hi = 0 means all M/2 modes.  Output: dev_out
 * [mode - mode_lo][point][rhs], complex128, modes u^s_n(x) with the same
 * normalisation as the densities (u^s(rho, theta, z) = (1/2pi) sum_n
 * e^{i n theta} u^s_n over n = -(M/2-1) .. M/2-1).  Allocates its scratch
 * (2 x points x N x modes complex) and synchronises the stream.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int  pmlbie_field(pmlbie_problem* prob, int n_pts, const double* rho, const double* z, const int* region,
                  int mode_lo, int mode_hi, int n_rhs, const void* dev_u1, const void* dev_phi1,
                  const void* dev_u2, const void* dev_phi2, void* dev_out, void* stream);

/* The same solve with HOST output buffers: the call copies the results to the
 * host (synchronising the stream).  Host buffers have the layout above. */
int  pmlbie_solve_host(pmlbie_problem* prob, int precision, int n_rhs, const double* polar,
                       double* u1, double* phi1, double* u2, double* phi2,
                       void* stream, pmlbie_report* rep);

/* Scan of count complex128 values in device memory for NaN or Inf (the
 * solves run it on their outputs).  Synchronises the stream.  Returns OK,
 * ENAN, EINVAL (NULL with count > 0) or ECUDA. */
int  pmlbie_check_finite(const void* dev, size_t count, void* stream);

/* Self-test of the device-side bounded waits (the tensor-core LU update waits
 * on an mbarrier with an iteration limit): one warp polls an mbarrier that no
 * thread arrives at, at most `iterations` times (1 .. 2^24), and reports the
 * expiry the way the update does.  Returns ETIMEOUT when the wait expired (the
 * expected outcome), OK if it completed, EINVAL, ECUDA.  The context stays
 * usable.  Synchronises the stream. */
int  pmlbie_selftest_wait(long long iterations, void* stream);

/* Self-test of the library's own elementary functions (not an operation of
 * the paper: the sampling loops of Sec. 3.1 / 4.1 evaluate e^{iq} with their
 * own exp, sin / cos and 1/sqrt).  Evaluates, at the n doubles of device
 * array dev_x, into device array dev_out:
 *   fn 0: exp(x)            -> out[i]   (arguments are clamped to [-708, 709])
 *   fn 1: sin(x), cos(x)    -> out[2 i], out[2 i + 1]
 *   fn 2: 1/sqrt(x)         -> out[i]   (x > 0)
 *   fn 10, 11, 12: the same by the CUDA math library (exp, sincos, rsqrt),
 *   the references the tests compare with.
 * dev_out holds n (fn 0, 2, 10, 12) or 2 n (fn 1, 11) doubles.  Synchronises
 * the stream.  EINVAL for an unknown fn, NULL buffers or n > 2^31; ECUDA. */
int  pmlbie_selftest_elementary(int fn, const void* dev_x, void* dev_out, size_t n, void* stream);

/* Pipe-throughput probe (not an operation of the paper: the measured
 * denominators of the library's roofline fractions).  kind 0: FP64 FMA
 * (independent fma chains on every SM), 1: FP32 FMA, 2: TF32 tensor cores
 * (tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, back to back from one
 * thread per SM, the accumulator in tensor memory).  *tflops receives the
 * rate of one timed launch after a warm-up launch (fused multiply-add = 2
 * flops).  Synchronises the stream; allocates 4 KB of device scratch.
 * EINVAL, ECUDA, ETIMEOUT (the tensor-core wait expired). */
int  pmlbie_selftest_peak(int kind, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PMLBIE_H */
