// Allocation-free variant of pmlbie_modal_kernels.
//
// Some callers cannot call cudaMalloc while they use this library: code that
// runs while another component owns every allocation (a framework with its own
// caching allocator and a fixed memory budget, or an embedding that forbids
// driver allocations after start-up).  This entry point computes the same
// modal kernels as pmlbie_modal_kernels, but keeps its close-pair scratch (the
// modal Laplace kernels of every close pair and their split modal values) in
// one file-scope device array of fixed size instead of allocating it.  The
// caller passes the problem (whose tables are already on the device) and the
// output buffer.
#include <mutex>

#include "internal.h"

namespace pmlbie {
namespace {

// Scratch shared by every call on a device: 64 MiB, held by each device that
// loads the library until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once per device
// (the host-side symbol is a stand-in, not a device address).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

int scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(PMLBIE_ENODEV, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(PMLBIE_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PMLBIE_OK;
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace pmlbie

using namespace pmlbie;

extern "C" int pmlbie_modal_kernels_noalloc(pmlbie_problem* prob, int mode_lo, int mode_hi, void* dev_out,
                                            void* stream) {
    if (!prob || !dev_out) return fail(PMLBIE_EINVAL, "problem or output NULL");
    const int nm = prob->P.M / 2;
    if (mode_lo < 0 || mode_hi > nm || mode_lo >= mode_hi) return fail(PMLBIE_EINVAL, "bad mode range");
    const size_t np = prob->H.near.size() ? prob->H.near.size() : 1;
    const size_t zd_bytes = round256(sizeof(double2) * np * 2 * prob->P.M);
    const size_t out_bytes = round256(sizeof(double2) * np * 4 * (size_t)(mode_hi - mode_lo));
    if (zd_bytes + out_bytes > kNoAllocScratchBytes)
        return fail(PMLBIE_EINVAL, "close-pair scratch needs " + std::to_string(zd_bytes + out_bytes) +
                                       " bytes, above the fixed " + std::to_string(kNoAllocScratchBytes) +
                                       "-byte array of the allocation-free call (fewer modes or a smaller "
                                       "problem fit)");
    if (!device_ready(prob))
        return fail(PMLBIE_EINVAL, "problem tables are not on the device yet: the allocation-free call needs a "
                                   "prior pmlbie_modal_kernels or pmlbie_solve on this problem");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != prob->device)
        return fail(PMLBIE_EINVAL, "current device is not the problem's device");
    void* base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    double2* zd = static_cast<double2*>(base);
    double2* nout = reinterpret_cast<double2*>(static_cast<char*>(base) + zd_bytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FarLaunch fl{mode_lo, mode_hi, nullptr, static_cast<double2*>(dev_out)};
    cudaError_t e = launch_far(prob, fl, s);
    if (e == cudaSuccess) e = launch_near(prob, mode_lo, mode_hi, zd, nout, s);
    if (e == cudaSuccess) e = launch_near_to_raw(prob, mode_lo, mode_hi, nout, static_cast<double2*>(dev_out), s);
    if (e != cudaSuccess) return fail(PMLBIE_ECUDA, std::string("modal kernels (no-alloc): ") + cudaGetErrorString(e));
    return PMLBIE_OK;
}
