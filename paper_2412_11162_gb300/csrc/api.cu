// C ABI of the PML-BIE modal solver: problem creation (host tables), device
// upload, modal kernels and the full solve.  See include/pmlbie.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>
#include <thread>

#include "internal.h"

using namespace pmlbie;

namespace {

constexpr double kPi = 3.14159265358979323846;

bool is_2a3b(int M) {
    if (M <= 0) return false;
    while (M % 2 == 0) M /= 2;
    while (M % 3 == 0) M /= 3;
    return M == 1;
}

template <typename T>
int upload(T*& dst, const std::vector<T>& src) {
    if (src.empty()) {
        dst = nullptr;
        return PMLBIE_OK;
    }
    PMLBIE_CUDA_TRY(cudaMalloc(&dst, sizeof(T) * src.size()));
    PMLBIE_CUDA_TRY(cudaMemcpy(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return PMLBIE_OK;
}

std::vector<double2> to_d2(const std::vector<cd>& v) {
    std::vector<double2> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = make_double2(v[i].real(), v[i].imag());
    return o;
}

}  // namespace

// device-side per-node extras live next to the problem (not in DeviceTables,
// which the kernels receive by value)
// The batched LU of one workspace (sizes and buffers fixed) as a CUDA graph:
// its 3 n / 32 + 1 dependent launches are replayed with one graph launch.
// The factorisation's sizes and buffers: a captured graph serves one key.
struct LuKey {
    int precision = -1, n = 0, batch = 0;
    const void *A = nullptr, *piv = nullptr, *info = nullptr, *img = nullptr, *ptab = nullptr;
    bool operator==(const LuKey& o) const {
        return precision == o.precision && n == o.n && batch == o.batch && A == o.A && piv == o.piv &&
               info == o.info && img == o.img && ptab == o.ptab;
    }
};

struct LuGraph {
    cudaGraphExec_t exec = nullptr;
    LuKey key;                  // of exec
    LuKey pending;              // of the last factorisation run directly
    bool has_pending = false;
    long launches = 0;          // kernels in the graph
    bool unavailable = false;   // capture failed once: launch directly
};

struct pmlbie_dev_extra {
    double *nu_r = nullptr, *nu_z = nullptr, *speed = nullptr;
    bool ready = false;
    cudaStream_t capture = nullptr;   // private stream the graph is captured on
    LuGraph lu;
    // event pairs around the LU's trailing-update launches (recorded by the
    // captured graph, or by a direct factorisation) and the pairs recorded
    // by the last factorisation
    std::vector<cudaEvent_t> upd_ev;
    int upd_pairs = 0;
    // high-priority stream of the close-pair chain beside the far kernel, and
    // the fork / join events of the system build
    cudaStream_t near_stream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // the complex64 factorisation's side stream (A' images beside the row swaps)
    LuSide lu_side;
};

namespace {

pmlbie_dev_extra* extra_of(pmlbie_problem* p) {
    static_assert(sizeof(void*) == sizeof(pmlbie_dev_extra*), "");
    return reinterpret_cast<pmlbie_dev_extra*>(p->ws_extra);
}

int ensure_device(pmlbie_problem* prob) {
    pmlbie_dev_extra* ex = extra_of(prob);
    if (ex->ready) return PMLBIE_OK;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(PMLBIE_ENODEV, "no CUDA device available");
    PMLBIE_CUDA_TRY(cudaGetDevice(&prob->device));
    const HostTables& H = prob->H;
    DeviceTables& D = prob->D;
    int rc;
    if ((rc = upload(D.rho, H.rho)) || (rc = upload(D.z, H.z)) || (rc = upload(D.I, H.I)) ||
        (rc = upload(D.Wu, H.Wu)) || (rc = upload(D.Wphi, H.Wphi)))
        return rc;
    std::vector<double2> rt = to_d2(H.rho_t), ncr = to_d2(H.nuc_r), ncz = to_d2(H.nuc_z);
    if ((rc = upload(D.rho_t, rt)) || (rc = upload(D.nuc_r, ncr)) || (rc = upload(D.nuc_z, ncz)) ||
        (rc = upload(D.cls, H.cls)) || (rc = upload(D.near, H.near)) || (rc = upload(D.near_lead, H.near_lead)) ||
        (rc = upload(D.bk, H.bk)) ||
        (rc = upload(D.off, H.off)) ||
        (rc = upload(D.corr_target, H.corr_target)) || (rc = upload(D.corr_m, H.corr_m)) ||
        (rc = upload(D.corr_coef, H.corr_coef)) || (rc = upload(D.Da, H.Da)) || (rc = upload(D.Db, H.Db)) ||
        (rc = upload(D.corr_start, H.corr_start)) || (rc = upload(D.corr_cmin, H.corr_cmin)) ||
        (rc = upload(D.corr_w, H.corr_w)))
        return rc;
    const int M = prob->P.M;
    std::vector<double2> cs(M / 2 + 1), tw(M), tw2(2 * M);
    for (int e = 0; e < 2 * M; ++e)
        tw2[e] = make_double2(std::cos(kPi * e / M), -std::sin(kPi * e / M));
    for (int j = 0; j <= M / 2; ++j) {
        double s = std::sin(kPi * j / M);
        cs[j] = make_double2(s * s, std::cos(2.0 * kPi * j / M));
    }
    for (int e = 0; e < M; ++e) tw[e] = make_double2(std::cos(2.0 * kPi * e / M), -std::sin(2.0 * kPi * e / M));
    if ((rc = upload(D.cos_tab, cs)) || (rc = upload(D.twid, tw)) || (rc = upload(D.twid2, tw2))) return rc;
    {
        const int nr = rec_table_len(M);
        std::vector<double2> up(nr), dn(nr);
        up[0] = dn[0] = make_double2(0.0, 0.0);
        for (int m = 1; m < nr; ++m) {
            up[m] = make_double2(4.0 * m / (2.0 * m + 1.0), (2.0 * m - 1.0) / (2.0 * m + 1.0));
            dn[m] = make_double2(4.0 * m / (2.0 * m - 1.0), (2.0 * m + 1.0) / (2.0 * m - 1.0));
        }
        if ((rc = upload(D.rec_up, up)) || (rc = upload(D.rec_dn, dn))) return rc;
    }
    {
        std::vector<float4> ftw, ftw2, fcs, ftrig;
        std::vector<float2> fexp, fwu(H.Wu.size()), fwp(H.Wphi.size());
        ff_tables(M, ftw, ftw2, fcs, fexp, ftrig);
        auto f2 = [](double x) {
            const float hi = (float)x;
            return make_float2(hi, (float)(x - (double)hi));
        };
        const double c4 = 0.5 / M;
        for (size_t m = 0; m < fwu.size(); ++m) {
            fwu[m] = f2(H.h * H.Wu[m] * c4);
            fwp[m] = f2(H.h * H.Wphi[m] * c4);
        }
        if ((rc = upload(D.twid_ff, ftw)) || (rc = upload(D.twid2_ff, ftw2)) || (rc = upload(D.cos_ff, fcs)) ||
            (rc = upload(D.exp_ff, fexp)) || (rc = upload(D.trig_ff, ftrig)) || (rc = upload(D.wuc_ff, fwu)) ||
            (rc = upload(D.wpc_ff, fwp)))
            return rc;
    }
    if ((rc = upload(ex->nu_r, H.nu_r)) || (rc = upload(ex->nu_z, H.nu_z)) || (rc = upload(ex->speed, H.speed)))
        return rc;
    ex->ready = true;
    return PMLBIE_OK;
}

void free_device(pmlbie_problem* prob) {
    DeviceTables& D = prob->D;
    void* ptrs[] = {D.rho, D.z, D.I, D.Wu, D.Wphi, D.rho_t, D.nuc_r, D.nuc_z, D.bk, D.off, D.cls, D.near, D.near_lead,
                    D.corr_target, D.corr_m, D.corr_coef, D.Da, D.Db, D.cos_tab, D.twid, D.twid2,
                    D.corr_start, D.corr_cmin, D.corr_w, D.rec_up, D.rec_dn, D.twid_ff, D.twid2_ff, D.cos_ff, D.exp_ff, D.trig_ff, D.wuc_ff,
                    D.wpc_ff};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    pmlbie_dev_extra* ex = extra_of(prob);
    if (ex) {
        if (ex->nu_r) cudaFree(ex->nu_r);
        if (ex->nu_z) cudaFree(ex->nu_z);
        if (ex->speed) cudaFree(ex->speed);
    }
    if (prob->ws) cudaFree(prob->ws);
    prob->ws = nullptr;
    if (ex && ex->lu.exec) cudaGraphExecDestroy(ex->lu.exec);
    if (ex && ex->capture) cudaStreamDestroy(ex->capture);
    if (ex && ex->near_stream) cudaStreamDestroy(ex->near_stream);
    if (ex && ex->fork) cudaEventDestroy(ex->fork);
    if (ex && ex->join) cudaEventDestroy(ex->join);
    if (ex && ex->lu_side.stream) cudaStreamDestroy(ex->lu_side.stream);
    if (ex && ex->lu_side.fork) cudaEventDestroy(ex->lu_side.fork);
    if (ex && ex->lu_side.join) cudaEventDestroy(ex->lu_side.join);
    if (ex) {
        ex->near_stream = nullptr;
        ex->fork = ex->join = nullptr;
        ex->lu_side = LuSide();
        for (cudaEvent_t e : ex->upd_ev) cudaEventDestroy(e);
        ex->upd_ev.clear();
        ex->upd_pairs = 0;
        ex->lu = LuGraph();
        ex->capture = nullptr;
    }
}

}  // namespace

bool pmlbie::device_ready(const pmlbie_problem* prob) {
    return prob && prob->ws_extra &&
           reinterpret_cast<const pmlbie_dev_extra*>(prob->ws_extra)->ready;
}

namespace {

// workspace carve-up of one solve
struct Workspace {
    double2 *A = nullptr, *zd = nullptr, *nout = nullptr, *b1 = nullptr, *b2 = nullptr, *B = nullptr,
            *X = nullptr, *R = nullptr;
    float2 *A32 = nullptr, *w32 = nullptr, *dinv = nullptr;
    unsigned char* img = nullptr;   // split operand images of the FP32 LU's trailing updates
    int2* ptab = nullptr;           // the FP32 LU's row-interchange mapping per step
    int *piv = nullptr, *info = nullptr, *active = nullptr, *nanflag = nullptr;
    double *rn = nullptr, *bn = nullptr, *xn = nullptr, *an = nullptr, *rpar = nullptr;
    size_t bytes = 0;
};

constexpr int kGmresM = 20;          // FGMRES restart length
constexpr int kGmresCycles = 10;     // FGMRES restarts at most
// a mode's refinement is done when, for every rhs, the relative residual
// |B - A x| / |B| <= kTolRel or the normwise backward error
// |B - A x| / (|A|_F |x| + |B|) <= kTolBwd, or when the backward error is
// below kTolFloor and stopped decreasing (the FP64 floor of ill-conditioned
// modes, whose |A| |x| >> |B|)
constexpr double kTolRel = 1e-13;
constexpr double kTolBwd = 1e-16;
constexpr double kTolFloor = 1e-14;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// nmodes: modes per chunk (every per-mode buffer holds one chunk)
Workspace plan(const pmlbie_problem* prob, int precision, int nrhs, int nmodes, char* base) {
    const size_t N = prob->P.N, M = prob->P.M, nm = nmodes, n2 = 2 * N;
    const size_t np = prob->H.near.size();
    Workspace w;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    w.A = (double2*)take(sizeof(double2) * nm * n2 * n2);
    if (precision == PMLBIE_MIXED) {
        w.A32 = (float2*)take(sizeof(float2) * nm * n2 * n2);
        w.w32 = (float2*)take(sizeof(float2) * nm * n2 * nrhs);
        // inverted 32 x 32 diagonal blocks of the factors (n2 / 32 of L and of U
        // per mode: 1/16 of the factor's bytes) for the correction solves
        if (n2 % 32 == 0) w.dinv = (float2*)take(sizeof(float2) * nm * diag_inv_elems((int)n2));
        w.img = (unsigned char*)take(lu_image_bytes((int)n2, (int)nm));
        w.ptab = (int2*)take(sizeof(int2) * lu_ptab_elems((int)n2, (int)nm));
        w.R = (double2*)take(sizeof(double2) * nm * n2 * nrhs);
    }
    w.zd = (double2*)take(near_zd_bytes(std::max<size_t>(np, 1), M, true));
    w.nout = (double2*)take(sizeof(double2) * std::max<size_t>(np, 1) * 4 * nm);
    w.b1 = (double2*)take(sizeof(double2) * nm * N * nrhs);
    w.b2 = (double2*)take(sizeof(double2) * nm * N * nrhs);
    w.B = (double2*)take(sizeof(double2) * nm * n2 * nrhs);
    w.X = (double2*)take(sizeof(double2) * nm * n2 * nrhs);
    w.piv = (int*)take(sizeof(int) * nm * n2);
    w.info = (int*)take(sizeof(int) * nm);
    w.nanflag = (int*)take(sizeof(int));
    w.active = (int*)take(sizeof(int) * nm);
    w.rn = (double*)take(sizeof(double) * nm * nrhs);
    w.bn = (double*)take(sizeof(double) * nm * nrhs);
    w.xn = (double*)take(sizeof(double) * nm * nrhs);
    w.an = (double*)take(sizeof(double) * nm);
    w.rpar = (double*)take(sizeof(double) * kRhsPar * nrhs);
    w.bytes = off;
    return w;
}

int get_workspace(pmlbie_problem* prob, int precision, int nrhs, int nmodes, Workspace& w) {
    Workspace sz = plan(prob, precision, nrhs, nmodes, nullptr);
    if (prob->ws_bytes < sz.bytes) {
        if (prob->ws) cudaFree(prob->ws);
        prob->ws = nullptr;
        prob->ws_bytes = 0;
        if (cudaMalloc(&prob->ws, sz.bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(PMLBIE_ENOMEM, "device workspace allocation failed (" + std::to_string(sz.bytes) + " bytes)");
        }
        prob->ws_bytes = sz.bytes;
    }
    w = plan(prob, precision, nrhs, nmodes, (char*)prob->ws);
    return PMLBIE_OK;
}

void fresnel(double w1, double w2, double phi, double* out6) {
    double kx = w1 * std::sin(phi);
    cd ks = (w2 > std::fabs(kx)) ? cd(std::sqrt(w2 * w2 - kx * kx), 0.0) : cd(0.0, std::sqrt(kx * kx - w2 * w2));
    cd R = 2.0 / (1.0 + ks / (w1 * std::cos(phi))) - 1.0;
    out6[0] = std::sin(phi);
    out6[1] = std::cos(phi);
    out6[2] = R.real();
    out6[3] = R.imag();
    out6[4] = ks.real();
    out6[5] = ks.imag();
}

// modal kernels + assembly into w.A for modes [lo, hi).  The far kernel and
// the close-pair chain (Laplace modes, float-float close pairs, FP64 PML close
// pairs) are independent until the assembly and load different pipes (the
// mixed path's far kernel the FP32 / integer issue, the PML pairs the FP64
// pipe): the chain runs on a high-priority stream forked from s, so that its
// CTAs are dispatched first and the far kernel's fill the SMs it leaves
// (mostly during the latency-bound Laplace-mode kernel); the assembly waits
// for both.  ev[0] = fork, ev[1] = far kernel done (on s), ev[4] / ev[5] =
// Laplace modes / float-float close pairs done and ev[2] = chain done (on the
// chain's stream), ev[6] = join, ev[3] = assembly done.
// (the mixed path samples the far pairs in float-float arithmetic when the
// problem's phases fit its range, else in FP64)
int build_system(pmlbie_problem* prob, int precision, Workspace& w, int lo, int hi, cudaStream_t s,
                 cudaEvent_t* ev) {
    FarLaunch fl{lo, hi, w.A, nullptr, true};
    pmlbie_dev_extra* ex = extra_of(prob);
    if (!ex->near_stream) {
        int least = 0, greatest = 0;
        PMLBIE_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        PMLBIE_CUDA_TRY(cudaStreamCreateWithPriority(&ex->near_stream, cudaStreamNonBlocking, greatest));
        PMLBIE_CUDA_TRY(cudaEventCreateWithFlags(&ex->fork, cudaEventDisableTiming));
        PMLBIE_CUDA_TRY(cudaEventCreateWithFlags(&ex->join, cudaEventDisableTiming));
    }
    const bool ff = precision == PMLBIE_MIXED && far_ff_supported(prob);
    cudaStream_t sn = ex->near_stream;
    PMLBIE_CUDA_TRY(cudaEventRecord(ev[0], s));
    PMLBIE_CUDA_TRY(cudaEventRecord(ex->fork, s));
    PMLBIE_CUDA_TRY(cudaStreamWaitEvent(sn, ex->fork, 0));
    // the far kernel first: its CTAs take the SMs the Laplace-mode kernel leaves idle
    PMLBIE_CUDA_TRY(ff ? launch_far_ff(prob, fl, s) : launch_far(prob, fl, s));
    PMLBIE_CUDA_TRY(cudaEventRecord(ev[1], s));
    PMLBIE_CUDA_TRY(launch_near(prob, lo, hi, w.zd, w.nout, sn, ev[4], ff, ev[5]));
    PMLBIE_CUDA_TRY(cudaEventRecord(ev[2], sn));
    PMLBIE_CUDA_TRY(cudaEventRecord(ex->join, sn));
    PMLBIE_CUDA_TRY(cudaStreamWaitEvent(s, ex->join, 0));
    PMLBIE_CUDA_TRY(cudaEventRecord(ev[6], s));
    PMLBIE_CUDA_TRY(launch_assemble(prob, lo, hi, w.nout, w.A, s));
    PMLBIE_CUDA_TRY(cudaEventRecord(ev[3], s));
    return PMLBIE_OK;
}

}  // namespace

extern "C" {

const char* pmlbie_last_error(void) { return error_text(); }

int pmlbie_create(const pmlbie_params* P, pmlbie_problem** out) {
    if (!out) return fail(PMLBIE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!P || P->struct_size < sizeof(pmlbie_params)) return fail(PMLBIE_EINVAL, "params NULL or struct_size too small");
    if (!(P->k1 > 0) || !(P->k2 > 0)) return fail(PMLBIE_EINVAL, "wavenumbers must be positive");
    if (!(P->a1 > 0) || !(P->T > 0) || !(P->S >= 0)) return fail(PMLBIE_EINVAL, "PML needs a1 > 0, T > 0, S >= 0");
    if (P->p < 2 || P->p > 16) return fail(PMLBIE_EINVAL, "p must be in [2, 16]");
    if (P->N < 32 || P->N > 16384) return fail(PMLBIE_EINVAL, "N must be in [32, 16384]");
    if (P->M < 16 || P->M > 768 || P->M % 4 || !is_2a3b(P->M))
        return fail(PMLBIE_EINVAL, "M must be 2^a 3^b, a multiple of 4, in [16, 768]");
    if (P->taylor_L < 3 || P->taylor_L > 7) return fail(PMLBIE_EINVAL, "taylor_L must be in [3, 7]");
    if (!(P->split_c > 0)) return fail(PMLBIE_EINVAL, "split_c must be positive");
    if (P->curve_kind == PMLBIE_CURVE_GAUSS_BUMP) {
        if (!(P->bump_R > 0) || !(P->bump_w > 0) || !(P->bump_R < P->a1))
            return fail(PMLBIE_EINVAL, "bump needs 0 < R < a1 and w > 0");
    } else if (P->curve_kind == PMLBIE_CURVE_WAVY_DENT) {
        if (!(P->wavy_R > 0) || !(P->wavy_R <= P->a1) || !(P->wavy_eps >= 0 && P->wavy_eps < 1) ||
            P->wavy_m < 1 || P->wavy_m > 64)
            return fail(PMLBIE_EINVAL, "wavy dent needs 0 < R <= a1, 0 <= eps < 1, 1 <= m <= 64");
    } else if (P->curve_kind == PMLBIE_CURVE_POLYLINE) {
        if (P->n_vertices < 2 || !P->vertices) return fail(PMLBIE_EINVAL, "polyline needs >= 2 vertices");
        if (P->vertices[0] != 0.0) return fail(PMLBIE_EINVAL, "polyline must start on the axis (rho = 0)");
        for (int i = 0; i < P->n_vertices; ++i)
            if (P->vertices[2 * i] < 0 || P->vertices[2 * i] > P->a1 + P->T + 1e-12 ||
                (P->vertices[2 * i] > P->a1 && P->vertices[2 * i + 1] != 0.0))
                return fail(PMLBIE_EINVAL, "polyline vertices must lie in rho <= a1 (or on z = 0 in the PML)");
    } else {
        return fail(PMLBIE_EINVAL, "unknown curve kind");
    }
    pmlbie_problem* prob = new (std::nothrow) pmlbie_problem();
    if (!prob) return fail(PMLBIE_ENOMEM, "host allocation failed");
    prob->P = *P;
    if (P->curve_kind == PMLBIE_CURVE_POLYLINE)
        prob->vertices.assign(P->vertices, P->vertices + 2 * P->n_vertices);
    prob->P.vertices = nullptr;
    prob->eta_split = P->split_c * 2.0 * kPi / P->M;
    prob->ws_extra = new pmlbie_dev_extra();
    int rc;
    try {
        rc = build_tables(prob);
    } catch (const std::bad_alloc&) {
        rc = fail(PMLBIE_ENOMEM, "host allocation failed while building tables");
    }
    if (rc != PMLBIE_OK) {
        delete reinterpret_cast<pmlbie_dev_extra*>(prob->ws_extra);
        delete prob;
        return rc;
    }
    *out = prob;
    return PMLBIE_OK;
}

void pmlbie_destroy(pmlbie_problem* prob) {
    if (!prob) return;
    if (extra_of(prob)->ready) free_device(prob);
    delete reinterpret_cast<pmlbie_dev_extra*>(prob->ws_extra);
    delete prob;
}

int pmlbie_nodes(const pmlbie_problem* prob, double* rho, double* z, double* speed, double* t, int n) {
    if (!prob || n != prob->P.N) return fail(PMLBIE_EINVAL, "problem NULL or n != N");
    const HostTables& H = prob->H;
    if (rho) std::memcpy(rho, H.rho.data(), sizeof(double) * n);
    if (z) std::memcpy(z, H.z.data(), sizeof(double) * n);
    if (speed) std::memcpy(speed, H.speed.data(), sizeof(double) * n);
    if (t) std::memcpy(t, H.t.data(), sizeof(double) * n);
    return PMLBIE_OK;
}

int pmlbie_diagonal(const pmlbie_problem* prob, double* Da, double* Db, int n) {
    if (!prob || n != prob->P.N) return fail(PMLBIE_EINVAL, "problem NULL or n != N");
    if (Da) std::memcpy(Da, prob->H.Da.data(), sizeof(double) * n);
    if (Db) std::memcpy(Db, prob->H.Db.data(), sizeof(double) * n);
    return PMLBIE_OK;
}

int pmlbie_dims(const pmlbie_problem* prob, int* N, int* M) {
    if (!prob) return fail(PMLBIE_EINVAL, "problem NULL");
    if (N) *N = prob->P.N;
    if (M) *M = prob->P.M;
    return PMLBIE_OK;
}

int pmlbie_near_count(const pmlbie_problem* prob, int* n_grid_near, int* n_corr) {
    if (!prob) return fail(PMLBIE_EINVAL, "problem NULL");
    if (n_grid_near) *n_grid_near = prob->H.n_grid_near;
    if (n_corr) *n_corr = (int)prob->H.near.size() - prob->H.n_grid_near;
    return PMLBIE_OK;
}

int pmlbie_near_pairs(const pmlbie_problem* prob, int* tgt, int* src, int* flags, int* mirror, int n) {
    if (!prob) return fail(PMLBIE_EINVAL, "problem NULL");
    const auto& v = prob->H.near;
    if (n != (int)v.size()) return fail(PMLBIE_EINVAL, "n must equal the close-pair count");
    for (int i = 0; i < n; ++i) {
        if (tgt) tgt[i] = v[i].tgt;
        if (src) src[i] = v[i].src;
        if (flags) flags[i] = v[i].flags;
        if (mirror) mirror[i] = v[i].mirror;
    }
    return PMLBIE_OK;
}

int pmlbie_node_tables(const pmlbie_problem* prob, double* I, double* nuc_r, double* nuc_z, double* Wu,
                       double* Wphi, int n) {
    if (!prob) return fail(PMLBIE_EINVAL, "problem NULL");
    const auto& H = prob->H;
    if (n != prob->P.N) return fail(PMLBIE_EINVAL, "n must equal N");
    for (int l = 0; l < n; ++l) {
        if (I) I[l] = H.I[l];
        if (nuc_r) nuc_r[2 * l] = H.nuc_r[l].real(), nuc_r[2 * l + 1] = H.nuc_r[l].imag();
        if (nuc_z) nuc_z[2 * l] = H.nuc_z[l].real(), nuc_z[2 * l + 1] = H.nuc_z[l].imag();
        if (Wu) Wu[l] = H.Wu[l];
        if (Wphi) Wphi[l] = H.Wphi[l];
    }
    return PMLBIE_OK;
}

int pmlbie_corrections(const pmlbie_problem* prob, int* target, double* tau, int* m, double* coef, int n) {
    if (!prob) return fail(PMLBIE_EINVAL, "problem NULL");
    const auto& H = prob->H;
    static_assert(PMLBIE_STENCIL == kStencil, "stencil width of the ABI");
    if (n != (int)H.corr_target.size()) return fail(PMLBIE_EINVAL, "n must equal the correction count");
    const size_t ns = (size_t)n * kStencil;
    if (target) std::memcpy(target, H.corr_target.data(), sizeof(int) * n);
    if (tau) std::memcpy(tau, H.corr_tau.data(), sizeof(double) * n);
    if (m) std::memcpy(m, H.corr_m.data(), sizeof(int) * ns);
    if (coef) std::memcpy(coef, H.corr_coef.data(), sizeof(double) * ns);
    return PMLBIE_OK;
}

int pmlbie_alpert_rule(int j, int a, double* x, double* w) {
    if (j < 2 || j > 12 || a < 1 || a > 16 || !x || !w) return fail(PMLBIE_EINVAL, "bad Alpert rule request");
    std::vector<double> xv, wv;
    try {
        alpert_log_rule(j, a, xv, wv);
    } catch (const std::exception& e) {
        return fail(PMLBIE_EINVAL, e.what());
    }
    std::memcpy(x, xv.data(), sizeof(double) * j);
    std::memcpy(w, wv.data(), sizeof(double) * j);
    return PMLBIE_OK;
}

size_t pmlbie_workspace_bytes(const pmlbie_problem* prob, int precision, int n_rhs) {
    if (!prob || n_rhs < 1) return 0;
    return plan(prob, precision, n_rhs, prob->P.M / 2, nullptr).bytes;
}

int pmlbie_modal_kernels(pmlbie_problem* prob, int mode_lo, int mode_hi, void* dev_out, void* stream) {
    return pmlbie_modal_kernels_ex(prob, PMLBIE_FP64, mode_lo, mode_hi, dev_out, stream);
}

int pmlbie_close_pair_kernels(pmlbie_problem* prob, int precision, int mode_lo, int mode_hi, void* dev_out,
                              void* stream) {
    if (!prob || !dev_out) return fail(PMLBIE_EINVAL, "problem or output NULL");
    if (precision != PMLBIE_FP64 && precision != PMLBIE_MIXED) return fail(PMLBIE_EINVAL, "bad precision");
    const int nm = prob->P.M / 2;
    if (mode_lo < 0 || mode_hi > nm || mode_lo >= mode_hi) return fail(PMLBIE_EINVAL, "bad mode range");
    int rc = ensure_device(prob);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = std::max<size_t>(prob->H.near.size(), 1);
    double2* zd = nullptr;
    PMLBIE_CUDA_TRY(cudaMalloc(&zd, near_zd_bytes(np, prob->P.M, true)));
    cudaError_t e = launch_near(prob, mode_lo, mode_hi, zd, (double2*)dev_out, s, nullptr,
                                precision == PMLBIE_MIXED && far_ff_supported(prob));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(zd);
    if (e != cudaSuccess) return fail(PMLBIE_ECUDA, std::string("close-pair kernels: ") + cudaGetErrorString(e));
    return PMLBIE_OK;
}

int pmlbie_modal_kernels_ex(pmlbie_problem* prob, int precision, int mode_lo, int mode_hi, void* dev_out,
                            void* stream) {
    if (!prob || !dev_out) return fail(PMLBIE_EINVAL, "problem or output NULL");
    if (precision != PMLBIE_FP64 && precision != PMLBIE_MIXED) return fail(PMLBIE_EINVAL, "bad precision");
    const int nm = prob->P.M / 2;
    if (mode_lo < 0 || mode_hi > nm || mode_lo >= mode_hi) return fail(PMLBIE_EINVAL, "bad mode range");
    int rc = ensure_device(prob);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = std::max<size_t>(prob->H.near.size(), 1);
    const int M = prob->P.M;
    double2 *zd = nullptr, *nout = nullptr;
    PMLBIE_CUDA_TRY(cudaMalloc(&zd, near_zd_bytes(np, M, true)));
    if (cudaMalloc(&nout, sizeof(double2) * np * 4 * (mode_hi - mode_lo)) != cudaSuccess) {
        cudaFree(zd);
        return fail(PMLBIE_ENOMEM, "scratch allocation failed");
    }
    FarLaunch fl{mode_lo, mode_hi, nullptr, (double2*)dev_out, true};
    cudaError_t e = precision == PMLBIE_MIXED && far_ff_supported(prob) ? launch_far_ff(prob, fl, s)
                                                                        : launch_far(prob, fl, s);
    if (e == cudaSuccess)
        e = launch_near(prob, mode_lo, mode_hi, zd, nout, s, nullptr, precision == PMLBIE_MIXED && far_ff_supported(prob));
    if (e == cudaSuccess) e = launch_near_to_raw(prob, mode_lo, mode_hi, nout, (double2*)dev_out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(zd);
    cudaFree(nout);
    if (e != cudaSuccess) return fail(PMLBIE_ECUDA, std::string("modal kernels: ") + cudaGetErrorString(e));
    return PMLBIE_OK;
}

// Batched LU of the workspace's matrices through the cached graph: captured
// on the problem's private stream the first time (or when the sizes or
// buffers change), then replayed on s.  Falls back to direct launches when
// the capture is refused.
// flag = 1 if any of the count doubles is NaN or Inf
__global__ void nonfinite_kernel(const double* v, size_t count, int* flag) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) {
            *flag = 1;
            return;
        }
}

static cudaError_t launch_nonfinite(const void* dev, size_t count_c128, int* flag, cudaStream_t s) {
    const size_t count = 2 * count_c128;
    const unsigned blocks = (unsigned)std::min<size_t>((count + 255) / 256, 152 * 8);
    if (blocks) nonfinite_kernel<<<blocks, 256, 0, s>>>((const double*)dev, count, flag);
    count_launch();
    return cudaGetLastError();
}

// Self-test of the bounded mbarrier wait: a barrier no thread arrives at.
__global__ void wait_probe_kernel(long long iters, int* expired) {
    __shared__ uint64_t bar;
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(addr));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t done = 0;
    for (long long it = 0; it < iters && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(addr), "r"(0u)
            : "memory");
    }
    if (threadIdx.x == 0) *expired = done ? 0 : 1;
}

// LU factorisations replayed from a graph by this thread's current call
thread_local int g_lu_graph_replays = 0;

static cudaError_t lu_direct(int precision, int n, int batch, void* A, int* piv, int* info, unsigned char* img,
                             int2* ptab, const LuSide* side, cudaStream_t s, cudaEvent_t* upd_ev = nullptr) {
    return precision == PMLBIE_FP64
               ? batched_lu<double2>(n, batch, (double2*)A, piv, info, s, nullptr, nullptr, nullptr, upd_ev)
               : batched_lu<float2>(n, batch, (float2*)A, piv, info, s, img, ptab, side, upd_ev);
}

// 2 x ceil(n / 32) timing events of the trailing updates; the pairs used are
// those of steps with a trailing matrix (n / 32 rounded up, minus one)
static cudaError_t ensure_update_events(pmlbie_dev_extra* ex, int n) {
    const size_t need = 2 * (size_t)((n + 31) / 32);
    while (ex->upd_ev.size() < need) {
        cudaEvent_t e = nullptr;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        ex->upd_ev.push_back(e);
    }
    ex->upd_pairs = (n + 31) / 32 - 1;
    return cudaSuccess;
}

static int batched_lu_graphed(pmlbie_problem* prob, int precision, int n, int batch, void* A, int* piv, int* info,
                              unsigned char* img, int2* ptab, cudaStream_t s) {
    pmlbie_dev_extra* ex = extra_of(prob);
    LuGraph& g = ex->lu;
    PMLBIE_CUDA_TRY(ensure_update_events(ex, n));
    if (!ex->lu_side.stream) {
        PMLBIE_CUDA_TRY(cudaStreamCreateWithFlags(&ex->lu_side.stream, cudaStreamNonBlocking));
        PMLBIE_CUDA_TRY(cudaEventCreateWithFlags(&ex->lu_side.fork, cudaEventDisableTiming));
        PMLBIE_CUDA_TRY(cudaEventCreateWithFlags(&ex->lu_side.join, cudaEventDisableTiming));
    }
    if (g.unavailable) {
        PMLBIE_CUDA_TRY(lu_direct(precision, n, batch, A, piv, info, img, ptab, &ex->lu_side, s, ex->upd_ev.data()));
        return PMLBIE_OK;
    }
    LuKey key;
    key.precision = precision;
    key.n = n;
    key.batch = batch;
    key.A = A;
    key.piv = piv;
    key.info = info;
    key.img = img;
    key.ptab = ptab;
    if (!(g.exec && g.key == key)) {
        // the first factorisation with these buffers runs directly (a one-off
        // solve does not pay for a capture); the second one is captured
        if (!(g.has_pending && g.pending == key)) {
            g.pending = key;
            g.has_pending = true;
            PMLBIE_CUDA_TRY(lu_direct(precision, n, batch, A, piv, info, img, ptab, &ex->lu_side, s, ex->upd_ev.data()));
            return PMLBIE_OK;
        }
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = LuGraph();
        if (!ex->capture) PMLBIE_CUDA_TRY(cudaStreamCreateWithFlags(&ex->capture, cudaStreamNonBlocking));
        PMLBIE_CUDA_TRY(precision == PMLBIE_FP64 ? lu_prepare<double2>() : lu_prepare<float2>());
        const long before = g_launches;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(ex->capture, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t el =
                lu_direct(precision, n, batch, A, piv, info, img, ptab, &ex->lu_side, ex->capture, ex->upd_ev.data());
            e = cudaStreamEndCapture(ex->capture, &graph);
            if (el != cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        const long captured = g_launches - before;   // kernels recorded into the graph
        g_launches = before;
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g = LuGraph();
            g.unavailable = true;
            PMLBIE_CUDA_TRY(lu_direct(precision, n, batch, A, piv, info, img, ptab, &ex->lu_side, s, ex->upd_ev.data()));
            return PMLBIE_OK;
        }
        g.launches = captured;
        g.key = key;
    }
    PMLBIE_CUDA_TRY(cudaGraphLaunch(g.exec, s));
    count_launch(g.launches);
    ++g_lu_graph_replays;
    return PMLBIE_OK;
}

// Accumulated device times and refinement statistics of a solve.
struct SolveStats {
    double ms_kernels = 0, ms_lu = 0, ms_solve = 0, ms_far = 0, ms_near = 0, ms_near_laplace = 0, ms_assemble = 0,
           ms_near_ff = 0, ms_lu_update = 0;
    int lu_update_launches = 0;
    int iters = 0;
    double resid = 0;
    int gmres_iters = 0, gmres_modes = 0;
    double bwd = 0;
    bool unconverged = false;
};

// One chunk of modes [lo, hi): system, RHS, LU, solve (+ refinement), outputs
// into u1.. (already offset to the chunk).  Synchronises the stream at the end.
static int solve_chunk(pmlbie_problem* prob, int precision, int n_rhs, bool point, int lo, int hi, Workspace& w,
                       double2* u1, double2* phi1, double2* u2, double2* phi2, cudaStream_t s, SolveStats& st) {
    const int N = prob->P.N, nm = hi - lo, n2 = 2 * N;
    cudaEvent_t ev[4], sev[7];
    for (auto& e : ev) PMLBIE_CUDA_TRY(cudaEventCreate(&e));
    for (auto& e : sev) PMLBIE_CUDA_TRY(cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t* e;
        cudaEvent_t* f;
        ~EvGuard() {
            for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]);
            for (int i = 0; i < 7; ++i) cudaEventDestroy(f[i]);
        }
    } guard{ev, sev};
    pmlbie_dev_extra* ex = extra_of(prob);
    int rc;
    PMLBIE_CUDA_TRY(cudaEventRecord(ev[0], s));
    if ((rc = build_system(prob, precision, w, lo, hi, s, sev))) return rc;
    // mixed: the right-hand sides (the FP64 block product, FP64-pipe bound) are
    // formed on s beside the complex64 conversion and factorisation, which run
    // on the high-priority stream and read / write only the FP32 copy; they
    // join before the refinement.  FP64: the factorisation overwrites w.A, so
    // the right-hand sides come first.
    const bool side = precision == PMLBIE_MIXED;
    cudaStream_t slu = side ? ex->near_stream : s;
    if (side) {
        PMLBIE_CUDA_TRY(cudaEventRecord(ev[1], s));
        PMLBIE_CUDA_TRY(cudaEventRecord(ex->fork, s));
        PMLBIE_CUDA_TRY(cudaStreamWaitEvent(slu, ex->fork, 0));
    }
    if (point)
        PMLBIE_CUDA_TRY(launch_point_rhs(prob, n_rhs, lo, hi, w.rpar, ex->speed, w.b1, w.b2, s));
    else
        PMLBIE_CUDA_TRY(launch_rhs(prob, n_rhs, lo, hi, w.rpar, ex->nu_r, ex->nu_z, ex->speed, w.b1, w.b2, s));
    PMLBIE_CUDA_TRY(launch_block_rhs(prob, n_rhs, nm, w.A, w.b1, w.b2, w.B, s));
    if (!side) PMLBIE_CUDA_TRY(cudaEventRecord(ev[1], s));
    PMLBIE_CUDA_TRY(cudaMemsetAsync(w.info, 0, sizeof(int) * nm, slu));
    const size_t xbytes = sizeof(double2) * (size_t)nm * n2 * n_rhs;
    int iters = 0;
    double resid = 0.0, bwd = 0.0;
    bool unconverged = false;
    std::vector<double> mres(nm, 0.0), mbwd(nm, 0.0);
    if (precision == PMLBIE_FP64) {
        if ((rc = batched_lu_graphed(prob, PMLBIE_FP64, n2, nm, w.A, w.piv, w.info, nullptr, nullptr, s))) return rc;
        PMLBIE_CUDA_TRY(cudaEventRecord(ev[2], s));
        PMLBIE_CUDA_TRY(cudaMemcpyAsync(w.X, w.B, xbytes, cudaMemcpyDeviceToDevice, s));
        PMLBIE_CUDA_TRY((batched_lu_solve<double2, double2>(n2, nm, n_rhs, w.A, w.piv, w.X, s)));
    } else {
        PMLBIE_CUDA_TRY(convert_fro2_c128(n2, nm, w.A, w.A32, w.an, slu));
        if ((rc = batched_lu_graphed(prob, PMLBIE_MIXED, n2, nm, w.A32, w.piv, w.info, w.img, w.ptab, slu)))
            return rc;
        if (w.dinv) PMLBIE_CUDA_TRY(batched_diag_inv(n2, nm, w.A32, w.dinv, slu));
        PMLBIE_CUDA_TRY(cudaEventRecord(ev[2], slu));
        PMLBIE_CUDA_TRY(cudaEventRecord(ex->join, slu));
        PMLBIE_CUDA_TRY(cudaStreamWaitEvent(s, ex->join, 0));
        PMLBIE_CUDA_TRY(cudaMemsetAsync(w.X, 0, xbytes, s));
        PMLBIE_CUDA_TRY(cudaMemcpyAsync(w.R, w.B, xbytes, cudaMemcpyDeviceToDevice, s));
        // refinement: FP64 residual with the FP64 matrix, FP32 correction solve; modes whose
        // residual is already below the tolerance for every rhs are left alone.  Modes whose
        // residual stops contracting (condition number x FP32 LU error near or above 1) are
        // restarted from zero and solved by FGMRES preconditioned with the same LU.
        std::vector<double> rn((size_t)nm * n_rhs), bn((size_t)nm * n_rhs), xn((size_t)nm * n_rhs), an(nm),
            prev(nm, 0.0), first(nm, 0.0);
        std::vector<int> act(nm, 1), slow(nm, 0);
        const int max_ir = 12;
        PMLBIE_CUDA_TRY(cudaMemcpyAsync(an.data(), w.an, sizeof(double) * nm, cudaMemcpyDeviceToHost, s));
        PMLBIE_CUDA_TRY(cudaMemcpyAsync(w.active, act.data(), sizeof(int) * nm, cudaMemcpyHostToDevice, s));
        for (iters = 0; iters <= max_ir; ++iters) {
            if (iters > 0) {
                PMLBIE_CUDA_TRY(residual_c128(n2, nm, n_rhs, w.A, w.X, w.B, w.R, w.rn, w.bn, w.xn, s, w.active));
                PMLBIE_CUDA_TRY(cudaMemcpyAsync(rn.data(), w.rn, sizeof(double) * rn.size(), cudaMemcpyDeviceToHost, s));
                PMLBIE_CUDA_TRY(cudaMemcpyAsync(bn.data(), w.bn, sizeof(double) * bn.size(), cudaMemcpyDeviceToHost, s));
                PMLBIE_CUDA_TRY(cudaMemcpyAsync(xn.data(), w.xn, sizeof(double) * xn.size(), cudaMemcpyDeviceToHost, s));
                PMLBIE_CUDA_TRY(cudaStreamSynchronize(s));
                int nact = 0;
                for (int mo = 0; mo < nm; ++mo) {
                    if (!act[mo]) continue;
                    double worst = 0.0, wbwd = 0.0;
                    bool ok = true;
                    for (int r = 0; r < n_rhs; ++r) {
                        const size_t i = (size_t)mo * n_rhs + r;
                        const double rr = std::sqrt(rn[i]), bb = std::sqrt(bn[i]);
                        const double den = std::sqrt(an[mo]) * std::sqrt(xn[i]) + bb;
                        const double rel = bb > 0 ? rr / bb : 0.0, bwd = den > 0 ? rr / den : 0.0;
                        worst = std::max(worst, rel);
                        wbwd = std::max(wbwd, bwd);
                        if (!(rel <= kTolRel || bwd <= kTolBwd)) ok = false;
                    }
                    mres[mo] = worst;
                    mbwd[mo] = wbwd;
                    const bool stalled = iters >= 2 && !(wbwd < 0.5 * prev[mo]);
                    if (ok || (stalled && wbwd <= kTolFloor)) {
                        act[mo] = 0;     // done, or at the FP64 floor
                    } else if (stalled) {
                        act[mo] = 0;     // contraction too slow or divergent: FGMRES
                        slow[mo] = 1;
                    } else {
                        ++nact;
                    }
                    prev[mo] = wbwd;
                    if (iters == 1) first[mo] = wbwd;
                }
                if (nact == 0) break;
                if (iters == max_ir) {
                    for (int mo = 0; mo < nm; ++mo)
                        if (act[mo]) act[mo] = 0, slow[mo] = 1;
                    break;
                }
                PMLBIE_CUDA_TRY(cudaMemcpyAsync(w.active, act.data(), sizeof(int) * nm, cudaMemcpyHostToDevice, s));
            }
            PMLBIE_CUDA_TRY(refine_step(n2, nm, n_rhs, w.A32, w.piv, w.R, w.w32, w.X, s, w.active, w.dinv, w.ptab));
        }
        const int nslow = (int)std::count(slow.begin(), slow.end(), 1);
        if (nslow > 0) {
            const size_t per = (size_t)n2 * n_rhs * sizeof(double2);
            for (int mo = 0; mo < nm; ++mo)
                // FGMRES starts from the refinement's last iterate when that
                // improved on the first one, else (divergence) from zero
                if (slow[mo] && !(mbwd[mo] < first[mo]))
                    PMLBIE_CUDA_TRY(cudaMemsetAsync((char*)w.X + per * mo, 0, per, s));
            int git = 0;
            // FGMRES on the contiguous range of modes [g0, g1) holding every
            // slow mode (its Krylov bases allocated for that range only)
            int g0 = nm, g1 = 0;
            for (int mo = 0; mo < nm; ++mo)
                if (slow[mo]) g0 = std::min(g0, mo), g1 = mo + 1;
            const int gn = g1 - g0;
            void* gm = nullptr;
            const size_t gbytes = gmres_scratch_bytes(n2, gn, n_rhs, kGmresM);
            if (cudaMalloc(&gm, gbytes) != cudaSuccess) {
                cudaGetLastError();
                return fail(PMLBIE_ENOMEM, "FGMRES scratch allocation failed (" + std::to_string(gbytes) + " bytes)");
            }
            std::vector<int> gslow(slow.begin() + g0, slow.begin() + g1);
            std::vector<double> gan(an.begin() + g0, an.begin() + g1), gres(mres.begin() + g0, mres.begin() + g1),
                gbwd(mbwd.begin() + g0, mbwd.begin() + g1);
            const size_t mat = (size_t)n2 * n2, vec = (size_t)n2 * n_rhs;
            rc = gmres_refine(n2, gn, n_rhs, w.A + g0 * mat, w.A32 + g0 * mat, w.piv + (size_t)g0 * n2,
                              w.B + g0 * vec, w.X + g0 * vec, gslow, w.active, gm, kGmresM, kGmresCycles, kTolRel,
                              kTolBwd, kTolFloor, gan, s, git, gres, gbwd,
                              w.dinv ? w.dinv + (size_t)g0 * diag_inv_elems(n2) : nullptr,
                              w.ptab + (size_t)g0 * lu_ptab_elems(n2, 1));
            cudaStreamSynchronize(s);
            cudaFree(gm);
            if (rc) return rc;
            for (int t = 0; t < gn; ++t) {
                slow[g0 + t] = gslow[t];
                mres[g0 + t] = gres[t];
                mbwd[g0 + t] = gbwd[t];
            }
            st.gmres_iters = std::max(st.gmres_iters, git);
            st.gmres_modes += nslow;
            for (int mo = 0; mo < nm; ++mo)
                if (slow[mo]) unconverged = true;    // still flagged: FGMRES missed the tolerance
        }
        resid = *std::max_element(mres.begin(), mres.end());
        bwd = *std::max_element(mbwd.begin(), mbwd.end());
    }
    PMLBIE_CUDA_TRY(launch_outputs(prob, n_rhs, nm, w.X, w.b1, w.b2, u1, phi1, u2, phi2, s));
    // NaN / Inf scan of the chunk's outputs
    PMLBIE_CUDA_TRY(cudaMemsetAsync(w.nanflag, 0, sizeof(int), s));
    const size_t per_out = (size_t)nm * N * n_rhs;
    for (double2* o : {u1, phi1, u2, phi2})
        if (o) PMLBIE_CUDA_TRY(launch_nonfinite(o, per_out, w.nanflag, s));
    PMLBIE_CUDA_TRY(cudaEventRecord(ev[3], s));
    PMLBIE_CUDA_TRY(cudaEventSynchronize(ev[3]));
    std::vector<int> info(nm);
    int nonfinite = 0;
    PMLBIE_CUDA_TRY(cudaMemcpy(info.data(), w.info, sizeof(int) * nm, cudaMemcpyDeviceToHost));
    PMLBIE_CUDA_TRY(cudaMemcpy(&nonfinite, w.nanflag, sizeof(int), cudaMemcpyDeviceToHost));
    // far kernel and close-pair chain from the fork (they overlap), assembly from the join
    float t[3], f[3], fl = 0.f;
    for (int i = 0; i < 3; ++i) cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]);
    cudaEventElapsedTime(&f[0], sev[0], sev[1]);
    cudaEventElapsedTime(&f[1], sev[0], sev[2]);
    cudaEventElapsedTime(&f[2], sev[6], sev[3]);
    cudaEventElapsedTime(&fl, sev[0], sev[4]);
    float fff = 0.f;
    cudaEventElapsedTime(&fff, sev[4], sev[5]);
    st.ms_near_ff += fff;
    for (int k = 0; k < ex->upd_pairs; ++k) {
        float tu = 0.f;
        if (cudaEventElapsedTime(&tu, ex->upd_ev[2 * k], ex->upd_ev[2 * k + 1]) == cudaSuccess) {
            st.ms_lu_update += tu;
            ++st.lu_update_launches;
        }
    }
    cudaGetLastError();
    st.ms_kernels += t[0];
    st.ms_lu += t[1];
    st.ms_solve += t[2];
    st.ms_far += f[0];
    st.ms_near += f[1];
    st.ms_assemble += f[2];
    st.ms_near_laplace += fl;
    st.iters = std::max(st.iters, iters);
    st.resid = std::max(st.resid, resid);
    st.bwd = std::max(st.bwd, bwd);
    st.unconverged = st.unconverged || unconverged;
    for (int i = 0; i < nm; ++i) {
        if (info[i] < 0)
            return fail(PMLBIE_ETIMEOUT, "tensor-core LU update did not complete (bounded wait expired) in mode " +
                                             std::to_string(lo + i));
        if (info[i]) return fail(PMLBIE_ESINGULAR, "zero pivot in mode " + std::to_string(lo + i));
    }
    if (nonfinite)
        return fail(PMLBIE_ENAN, "NaN or Inf in the outputs of modes " + std::to_string(lo) + ".." +
                                     std::to_string(hi - 1));
    return PMLBIE_OK;
}

int pmlbie_solve_ex(pmlbie_problem* prob, const pmlbie_solve_opts* o, void* dev_u1, void* dev_phi1,
                    void* dev_u2, void* dev_phi2, void* stream, pmlbie_report* rep) {
    if (!prob || !o || o->struct_size < sizeof(pmlbie_solve_opts)) return fail(PMLBIE_EINVAL, "bad problem or options");
    const int precision = o->precision, n_rhs = o->n_rhs, nmodes_all = prob->P.M / 2;
    const bool point = o->source_rho || o->source_z;
    if (n_rhs < 1 || n_rhs > 4096) return fail(PMLBIE_EINVAL, "n_rhs must be in [1, 4096]");
    if (point ? (o->polar || !o->source_rho || !o->source_z) : !o->polar)
        return fail(PMLBIE_EINVAL, "give either polar angles or source_rho and source_z");
    if (precision != PMLBIE_FP64 && precision != PMLBIE_MIXED) return fail(PMLBIE_EINVAL, "bad precision");
    for (int r = 0; r < n_rhs; ++r) {
        if (!point && !(o->polar[r] >= 0.0 && o->polar[r] < 0.5 * kPi))
            return fail(PMLBIE_EINVAL, "polar angle must be in [0, pi/2)");
        if (o->azimuth && !std::isfinite(o->azimuth[r])) return fail(PMLBIE_EINVAL, "azimuth must be finite");
    }
    if (point) {
        // sources in the physical region, far-pair separated from every node
        const double eta = prob->P.split_c * 2.0 * kPi / prob->P.M;
        for (int r = 0; r < n_rhs; ++r) {
            const double rs = o->source_rho[r], zs = o->source_z[r];
            if (!(rs >= 0.0 && rs < prob->P.a1) || !std::isfinite(zs))
                return fail(PMLBIE_EINVAL, "source must have 0 <= rho < a1 and finite z");
            for (size_t m = 0; m < prob->H.rho.size(); ++m) {
                const double dr = rs - prob->H.rho[m], dz = zs - prob->H.z[m];
                if (dr * dr + dz * dz < eta * eta * rs * prob->H.rho[m])
                    return fail(PMLBIE_EINVAL, "source " + std::to_string(r) +
                                                   " is too close to the interface for the M-point rule");
            }
        }
    }
    int lo = o->mode_lo, hi = o->mode_hi;
    if (lo == 0 && hi == 0) hi = nmodes_all;
    if (lo < 0 || hi > nmodes_all || lo >= hi) return fail(PMLBIE_EINVAL, "bad mode range");
    if (o->max_chunk_modes < 0) return fail(PMLBIE_EINVAL, "max_chunk_modes must be >= 0");
    int rc = ensure_device(prob);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // Waves that share a polar angle differ only by their azimuth, and mode n
    // of the solution rotates by e^{-i n azimuth} (Sec. 3.3 modes, plane-wave
    // data): solve the distinct polar angles at azimuth 0, then rotate.
    // Point sources that share (rho_s, z_s) likewise.
    std::vector<double> pu, pz;
    std::vector<int> idx(n_rhs);
    for (int r = 0; r < n_rhs; ++r) {
        const double k0 = point ? o->source_rho[r] : o->polar[r], k1 = point ? o->source_z[r] : 0.0;
        int k = 0;
        while (k < (int)pu.size() && !(pu[k] == k0 && pz[k] == k1)) ++k;
        if (k == (int)pu.size()) pu.push_back(k0), pz.push_back(k1);
        idx[r] = k;
    }
    if ((int)pu.size() < n_rhs) {
        const int nu = (int)pu.size(), nmo = hi - lo, N = prob->P.N;
        pmlbie_solve_opts o2 = *o;
        o2.n_rhs = nu;
        if (point) {
            o2.source_rho = pu.data();
            o2.source_z = pz.data();
        } else {
            o2.polar = pu.data();
        }
        o2.azimuth = nullptr;
        void* outs[4] = {dev_u1, dev_phi1, dev_u2, dev_phi2};
        void* tmp[4] = {nullptr, nullptr, nullptr, nullptr};
        int* d_idx = nullptr;
        double* d_az = nullptr;
        struct Free {
            void** t;
            int** i;
            double** a;
            ~Free() {
                for (int k = 0; k < 4; ++k)
                    if (t[k]) cudaFree(t[k]);
                if (*i) cudaFree(*i);
                if (*a) cudaFree(*a);
            }
        } fr{tmp, &d_idx, &d_az};
        const size_t tb = sizeof(double2) * (size_t)nmo * N * nu;
        for (int k = 0; k < 4; ++k)
            if (outs[k] && cudaMalloc(&tmp[k], tb) != cudaSuccess) {
                cudaGetLastError();
                return fail(PMLBIE_ENOMEM, "allocation of the distinct-wave outputs failed");
            }
        if (cudaMalloc(&d_idx, sizeof(int) * n_rhs) != cudaSuccess ||
            cudaMalloc(&d_az, sizeof(double) * n_rhs) != cudaSuccess) {
            cudaGetLastError();
            return fail(PMLBIE_ENOMEM, "allocation of the wave tables failed");
        }
        std::vector<double> az(n_rhs, 0.0);
        if (o->azimuth) az.assign(o->azimuth, o->azimuth + n_rhs);
        PMLBIE_CUDA_TRY(cudaMemcpyAsync(d_idx, idx.data(), sizeof(int) * n_rhs, cudaMemcpyHostToDevice, s));
        PMLBIE_CUDA_TRY(cudaMemcpyAsync(d_az, az.data(), sizeof(double) * n_rhs, cudaMemcpyHostToDevice, s));
        rc = pmlbie_solve_ex(prob, &o2, tmp[0], tmp[1], tmp[2], tmp[3], stream, rep);
        if (rc && rc != PMLBIE_ENOCONVERGE) return rc;
        const int rc_solve = rc;
        std::string msg = rc ? error_text() : "";
        for (int k = 0; k < 4; ++k)
            if (outs[k])
                PMLBIE_CUDA_TRY(launch_expand_waves(N, nmo, lo, nu, n_rhs, d_idx, d_az, (const double2*)tmp[k],
                                                    (double2*)outs[k], s));
        PMLBIE_CUDA_TRY(cudaStreamSynchronize(s));
        if (rep && rep->struct_size >= sizeof(pmlbie_report)) rep->launches += 4;
        return rc_solve ? fail(rc_solve, msg) : PMLBIE_OK;
    }
    // modes per chunk: the caller's cap, then the workspace limit (default: 90 %
    // of the free device memory plus the workspace the problem already holds)
    int chunk = hi - lo;
    if (o->max_chunk_modes > 0) chunk = std::min(chunk, o->max_chunk_modes);
    size_t limit = o->workspace_limit;
    if (limit == 0) {
        size_t fr = 0, tot = 0;
        PMLBIE_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        limit = (size_t)(0.9 * (double)(fr + prob->ws_bytes));
    }
    // the largest chunk whose workspace fits (binary search), then chunks of
    // equal size: each chunk re-samples the kernels, so the count is minimal
    if (plan(prob, precision, n_rhs, 1, nullptr).bytes > limit)
        return fail(PMLBIE_ENOMEM, "one mode's workspace exceeds the workspace limit");
    if (plan(prob, precision, n_rhs, chunk, nullptr).bytes > limit) {
        int ok = 1, bad = chunk;
        while (bad - ok > 1) {
            const int mid = ok + (bad - ok) / 2;
            (plan(prob, precision, n_rhs, mid, nullptr).bytes <= limit ? ok : bad) = mid;
        }
        const int nchunks = (hi - lo + ok - 1) / ok;
        chunk = (hi - lo + nchunks - 1) / nchunks;
    }
    Workspace w;
    if ((rc = get_workspace(prob, precision, n_rhs, chunk, w))) return rc;
    g_launches = 0;
    g_lu_graph_replays = 0;
    std::vector<double> rpar((size_t)kRhsPar * n_rhs, 0.0);
    for (int r = 0; r < n_rhs; ++r) {
        if (point) {
            rpar[(size_t)kRhsPar * r] = o->source_rho[r];
            rpar[(size_t)kRhsPar * r + 1] = o->source_z[r];
        } else {
            fresnel(prob->P.k1, prob->P.k2, o->polar[r], &rpar[(size_t)kRhsPar * r]);
        }
        rpar[(size_t)kRhsPar * r + 6] = o->azimuth ? o->azimuth[r] : 0.0;
    }
    PMLBIE_CUDA_TRY(cudaMemcpyAsync(w.rpar, rpar.data(), sizeof(double) * rpar.size(), cudaMemcpyHostToDevice, s));
    SolveStats st;
    const size_t per_mode = (size_t)prob->P.N * n_rhs;
    auto at = [&](void* p, int m) { return p ? (double2*)p + (size_t)(m - lo) * per_mode : nullptr; };
    int chunks = 0;
    for (int c0 = lo; c0 < hi; c0 += chunk) {
        const int c1 = std::min(hi, c0 + chunk);
        rc = solve_chunk(prob, precision, n_rhs, point, c0, c1, w, at(dev_u1, c0), at(dev_phi1, c0), at(dev_u2, c0),
                         at(dev_phi2, c0), s, st);
        ++chunks;
        if (rc) return rc;
    }
    if (rep && rep->struct_size >= sizeof(pmlbie_report)) {
        rep->n_modes = hi - lo;
        rep->near_pairs = (int)prob->H.near.size();
        rep->refine_iters = st.iters;
        rep->residual = st.resid;
        rep->ms_kernels = st.ms_kernels;
        rep->ms_lu = st.ms_lu;
        rep->ms_solve = st.ms_solve;
        rep->ms_far = st.ms_far;
        rep->ms_near = st.ms_near;
        rep->ms_assemble = st.ms_assemble;
        rep->ms_near_laplace = st.ms_near_laplace;
        rep->ms_near_ff = st.ms_near_ff;
        rep->ms_lu_update = st.ms_lu_update;
        rep->lu_update_launches = st.lu_update_launches;
        rep->launches = (int)g_launches;
        int* fc = prob->far_counts;
        if (fc[0] < 0) {
            const int N = prob->P.N;
            const auto far = [&](int l, int m) { return prob->H.cls[(size_t)l * N + m] == (uint8_t)kFar; };
            const auto phys = [&](int l) { return prob->H.I[l] == 0.0; };
            int n[4] = {0, 0, 0, 0};
            for (int l = 0; l < N; ++l)
                for (int m = 0; m < N; ++m) {
                    if (!far(l, m) && !far(m, l)) continue;
                    const bool pp = phys(l) && phys(m);
                    if (far(l, m)) n[0] += 1, n[1] += pp;
                    if (m < l) n[2] += 1, n[3] += pp;
                }
            for (int k = 0; k < 4; ++k) fc[k] = n[k];
        }
        rep->far_pairs = fc[0];
        rep->far_pairs_physical = fc[1];
        rep->far_pairs_sampled = fc[2];
        rep->far_pairs_sampled_physical = fc[3];
        rep->chunks = chunks;
        rep->chunk_modes = chunk;
        rep->gmres_modes = st.gmres_modes;
        rep->gmres_iters = st.gmres_iters;
        rep->backward_error = st.bwd;
        rep->lu_graph_replays = g_lu_graph_replays;
        rep->far_pairs_per_cta = g_far_pairs_per_cta;
        rep->ms_far_alone =
            precision == PMLBIE_MIXED && far_ff_supported(prob) ? far_ff_alone_ms(prob, chunk, false) : 0.0;
    }
    if (precision == PMLBIE_MIXED && st.unconverged)
        return fail(PMLBIE_ENOCONVERGE, "refinement missed its tolerance: residual " + std::to_string(st.resid) +
                                            ", backward error " + std::to_string(st.bwd));
    return PMLBIE_OK;
}

int pmlbie_solve(pmlbie_problem* prob, int precision, int n_rhs, const double* polar, void* dev_u1,
                 void* dev_phi1, void* dev_u2, void* dev_phi2, void* stream, pmlbie_report* rep) {
    pmlbie_solve_opts o;
    std::memset(&o, 0, sizeof(o));
    o.struct_size = sizeof(o);
    o.precision = precision;
    o.n_rhs = n_rhs;
    o.polar = polar;
    return pmlbie_solve_ex(prob, &o, dev_u1, dev_phi1, dev_u2, dev_phi2, stream, rep);
}

int pmlbie_solve_batch(pmlbie_problem* const* probs, int n_probs, const pmlbie_solve_opts* opts,
                       void* const* dev_u1, void* const* dev_phi1, void* const* dev_u2, void* const* dev_phi2,
                       int n_streams, int release_workspace, void* stream, pmlbie_report* reps) {
    if (!probs || n_probs < 1 || !opts) return fail(PMLBIE_EINVAL, "batch: bad problems or options");
    if (n_streams < 1 || n_streams > 8) return fail(PMLBIE_EINVAL, "batch: n_streams must be 1..8");
    for (int i = 0; i < n_probs; ++i) {
        if (!probs[i]) return fail(PMLBIE_EINVAL, "batch: NULL problem " + std::to_string(i));
        for (int j = 0; j < i; ++j)
            if (probs[j] == probs[i]) return fail(PMLBIE_EINVAL, "batch: a problem appears twice");
    }
    int dev = 0;
    PMLBIE_CUDA_TRY(cudaGetDevice(&dev));
    const int ns = std::min(n_streams, n_probs);
    cudaStream_t caller = (cudaStream_t)stream;
    std::vector<cudaStream_t> st(ns, nullptr);
    std::vector<cudaEvent_t> done(ns, nullptr);
    cudaEvent_t start = nullptr;
    struct Guard {
        std::vector<cudaStream_t>& s;
        std::vector<cudaEvent_t>& d;
        cudaEvent_t& st;
        ~Guard() {
            for (auto x : s)
                if (x) cudaStreamDestroy(x);
            for (auto x : d)
                if (x) cudaEventDestroy(x);
            if (st) cudaEventDestroy(st);
        }
    } guard{st, done, start};
    PMLBIE_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    PMLBIE_CUDA_TRY(cudaEventRecord(start, caller));
    for (int k = 0; k < ns; ++k) {
        PMLBIE_CUDA_TRY(cudaStreamCreateWithFlags(&st[k], cudaStreamNonBlocking));
        PMLBIE_CUDA_TRY(cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming));
        PMLBIE_CUDA_TRY(cudaStreamWaitEvent(st[k], start, 0));
    }
    // instance i runs on worker i mod ns; each worker is a host thread driving
    // its stream, so one instance's latency-bound phases overlap another's work
    std::vector<int> rc(n_probs, PMLBIE_OK);
    std::vector<std::string> msg(n_probs);
    auto work = [&](int k) {
        cudaSetDevice(dev);
        for (int i = k; i < n_probs; i += ns) {
            pmlbie_report* rep = reps ? reps + i : nullptr;
            auto at = [&](void* const* arr) { return arr ? arr[i] : nullptr; };
            rc[i] = pmlbie_solve_ex(probs[i], opts + i, at(dev_u1), at(dev_phi1), at(dev_u2), at(dev_phi2), st[k],
                                    rep);
            if (rc[i]) msg[i] = error_text();
            if (release_workspace) {
                cudaStreamSynchronize(st[k]);
                if (probs[i]->ws) cudaFree(probs[i]->ws);
                probs[i]->ws = nullptr;
                probs[i]->ws_bytes = 0;
            }
        }
        cudaEventRecord(done[k], st[k]);
    };
    std::vector<std::thread> th;
    for (int k = 1; k < ns; ++k) th.emplace_back(work, k);
    work(0);
    for (auto& t : th) t.join();
    for (int k = 0; k < ns; ++k) PMLBIE_CUDA_TRY(cudaStreamWaitEvent(caller, done[k], 0));
    for (int i = 0; i < n_probs; ++i)
        if (rc[i]) return fail(rc[i], "batch instance " + std::to_string(i) + ": " + msg[i]);
    return PMLBIE_OK;
}

int pmlbie_field(pmlbie_problem* prob, int n_pts, const double* rho, const double* z, const int* region, int mode_lo,
                 int mode_hi, int n_rhs, const void* dev_u1, const void* dev_phi1, const void* dev_u2,
                 const void* dev_phi2, void* dev_out, void* stream) {
    if (!prob || n_pts < 1 || !rho || !z || !region || !dev_out || n_rhs < 1)
        return fail(PMLBIE_EINVAL, "field: bad problem, points or output");
    const int nmodes_all = prob->P.M / 2;
    if (mode_lo == 0 && mode_hi == 0) mode_hi = nmodes_all;
    if (mode_lo < 0 || mode_hi > nmodes_all || mode_lo >= mode_hi) return fail(PMLBIE_EINVAL, "field: bad mode range");
    bool up = false, down = false;
    for (int p = 0; p < n_pts; ++p) {
        if (!(rho[p] >= 0.0 && rho[p] < prob->P.a1) || !std::isfinite(z[p]))
            return fail(PMLBIE_EINVAL, "field: points must have 0 <= rho < a1 (physical region)");
        if (region[p] != 0 && region[p] != 1) return fail(PMLBIE_EINVAL, "field: region must be 0 (upper) or 1 (lower)");
        (region[p] == 0 ? up : down) = true;
    }
    if ((up && (!dev_u1 || !dev_phi1)) || (down && (!dev_u2 || !dev_phi2)))
        return fail(PMLBIE_EINVAL, "field: densities of a medium holding points are missing");
    int rc = ensure_device(prob);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nm = (size_t)(mode_hi - mode_lo), N = prob->P.N;
    double *d_rho = nullptr, *d_z = nullptr;
    int* d_reg = nullptr;
    double2* coef = nullptr;
    struct Free {
        double** a;
        double** b;
        int** c;
        double2** d;
        ~Free() {
            if (*a) cudaFree(*a);
            if (*b) cudaFree(*b);
            if (*c) cudaFree(*c);
            if (*d) cudaFree(*d);
        }
    } fr{&d_rho, &d_z, &d_reg, &coef};
    if (cudaMalloc(&d_rho, sizeof(double) * n_pts) != cudaSuccess ||
        cudaMalloc(&d_z, sizeof(double) * n_pts) != cudaSuccess ||
        cudaMalloc(&d_reg, sizeof(int) * n_pts) != cudaSuccess ||
        cudaMalloc(&coef, sizeof(double2) * 2 * nm * N * n_pts) != cudaSuccess) {
        cudaGetLastError();
        return fail(PMLBIE_ENOMEM, "field: scratch allocation failed");
    }
    PMLBIE_CUDA_TRY(cudaMemcpyAsync(d_rho, rho, sizeof(double) * n_pts, cudaMemcpyHostToDevice, s));
    PMLBIE_CUDA_TRY(cudaMemcpyAsync(d_z, z, sizeof(double) * n_pts, cudaMemcpyHostToDevice, s));
    PMLBIE_CUDA_TRY(cudaMemcpyAsync(d_reg, region, sizeof(int) * n_pts, cudaMemcpyHostToDevice, s));
    PMLBIE_CUDA_TRY(launch_field(prob, n_pts, d_rho, d_z, d_reg, mode_lo, mode_hi, n_rhs, (const double2*)dev_u1,
                                 (const double2*)dev_phi1, (const double2*)dev_u2, (const double2*)dev_phi2, coef,
                                 (double2*)dev_out, s));
    PMLBIE_CUDA_TRY(cudaStreamSynchronize(s));
    return PMLBIE_OK;
}

int pmlbie_check_finite(const void* dev, size_t count, void* stream) {
    if (count == 0) return PMLBIE_OK;
    if (!dev) return fail(PMLBIE_EINVAL, "NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    int* flag = nullptr;
    if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(PMLBIE_ENOMEM, "flag allocation failed");
    }
    int h = 0;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_nonfinite(dev, count, flag, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flag);
    if (e != cudaSuccess) return fail(PMLBIE_ECUDA, std::string("finiteness scan: ") + cudaGetErrorString(e));
    return h ? fail(PMLBIE_ENAN, "NaN or Inf in the buffer") : PMLBIE_OK;
}

int pmlbie_selftest_wait(long long iterations, void* stream) {
    if (iterations < 1 || iterations > (1ll << 24)) return fail(PMLBIE_EINVAL, "iterations must be in [1, 2^24]");
    cudaStream_t s = (cudaStream_t)stream;
    int* flag = nullptr;
    if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(PMLBIE_ENOMEM, "flag allocation failed");
    }
    int h = 0;
    wait_probe_kernel<<<1, 32, 0, s>>>(iterations, flag);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flag);
    if (e != cudaSuccess) return fail(PMLBIE_ECUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
    return h ? fail(PMLBIE_ETIMEOUT, "bounded wait expired after " + std::to_string(iterations) + " polls")
             : PMLBIE_OK;
}

int pmlbie_selftest_peak(int kind, double* tflops, void* stream) {
    if (kind < 0 || kind > 2 || !tflops) return fail(PMLBIE_EINVAL, "kind must be 0, 1 or 2 and tflops non-NULL");
    return peak_probe(kind, tflops, static_cast<cudaStream_t>(stream));
}

int pmlbie_selftest_elementary(int fn, const void* dev_x, void* dev_out, size_t n, void* stream) {
    if (!elementary_selftest_known(fn) && !ff_elementary_known(fn))
        return fail(PMLBIE_EINVAL, "unknown elementary-function selector");
    if (n > 0 && (!dev_x || !dev_out)) return fail(PMLBIE_EINVAL, "NULL buffer");
    if (n > ((size_t)1 << 31)) return fail(PMLBIE_EINVAL, "n above 2^31");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (ff_elementary_known(fn)) {
        PMLBIE_CUDA_TRY(launch_ff_elementary(fn, static_cast<const double*>(dev_x), static_cast<double*>(dev_out), n, s));
        return PMLBIE_OK;
    }
    PMLBIE_CUDA_TRY(launch_elementary_selftest(fn, static_cast<const double*>(dev_x), static_cast<double*>(dev_out),
                                               n, s));
    PMLBIE_CUDA_TRY(cudaStreamSynchronize(s));
    return PMLBIE_OK;
}

int pmlbie_solve_host(pmlbie_problem* prob, int precision, int n_rhs, const double* polar, double* u1,
                      double* phi1, double* u2, double* phi2, void* stream, pmlbie_report* rep) {
    if (!prob || n_rhs < 1) return fail(PMLBIE_EINVAL, "bad problem or n_rhs");
    int rc = ensure_device(prob);
    if (rc) return rc;
    const size_t cnt = (size_t)(prob->P.M / 2) * prob->P.N * n_rhs;
    double* hosts[4] = {u1, phi1, u2, phi2};
    void* dev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int i = 0; i < 4; ++i)
        if (hosts[i] && cudaMalloc(&dev[i], sizeof(double2) * cnt) != cudaSuccess) {
            for (int k = 0; k < 4; ++k)
                if (dev[k]) cudaFree(dev[k]);
            return fail(PMLBIE_ENOMEM, "output allocation failed");
        }
    rc = pmlbie_solve(prob, precision, n_rhs, polar, dev[0], dev[1], dev[2], dev[3], stream, rep);
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < 4; ++i)
        if (hosts[i] && (rc == PMLBIE_OK || rc == PMLBIE_ENOCONVERGE))
            cudaMemcpyAsync(hosts[i], dev[i], sizeof(double2) * cnt, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    for (int i = 0; i < 4; ++i)
        if (dev[i]) cudaFree(dev[i]);
    if (e != cudaSuccess && rc == PMLBIE_OK) return fail(PMLBIE_ECUDA, cudaGetErrorString(e));
    return rc;
}

}  // extern "C"
