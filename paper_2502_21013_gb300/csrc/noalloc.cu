// Outer residual without any allocation by the library during the call.
//
// Some callers cannot let a library call cudaMalloc while they run: a
// framework whose own memory pool owns the whole device and forbids
// allocations it does not manage, a process with a hard device-memory budget
// where an allocation may fail at an arbitrary point, or a latency-critical
// loop that cannot afford the device-wide synchronisation cudaMalloc and
// cudaFree imply.  For them ptp_residual_noalloc_dev computes the same
// R = F - A(U) and ||R|| as ptp_residual_dev, but its scratch (the block
// partial sums of the norm, their ticket counter and the iron element fluxes)
// lives in the fixed array below instead of the context's allocations.
//
// The array is 4 MiB; every GPU that loads this library holds it until the
// process exits.  Every call shares it and it keeps the last call's
// contents, so two calls that overlap on the GPU (on different streams or
// from different contexts on the same device) race and corrupt each other.
#include <mutex>

#include "kernels.h"

namespace ptp {
namespace {

constexpr size_t kScratchDoubles = 524288;          // 4 MiB
constexpr size_t kCounterDoubles = 8;               // ticket counter (first 8 bytes used)
constexpr size_t kPartialDoubles = 2048;            // block partials of ||R||^2
constexpr size_t kFluxOffset = kCounterDoubles + kPartialDoubles;
constexpr size_t kMaxFluxDoubles = kScratchDoubles - kFluxOffset;  // Qx and Qy together

static __device__ __align__(256) double g_residual_scratch[kScratchDoubles];

// Device address of g_residual_scratch per device, looked up once.
std::mutex g_mutex;
void* g_addr[256] = {};

void* scratch_address(int device) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (device < 0 || device >= 256) throw Error(PTP_EINVAL, "device index out of range");
    if (!g_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_residual_scratch);  // the device is current
        if (e != cudaSuccess || !p)
            throw Error(PTP_ECUDA, std::string("cudaGetSymbolAddress of the residual scratch failed: ") +
                                       cudaGetErrorString(e));
        g_addr[device] = p;
    }
    return g_addr[device];
}

}  // namespace
}  // namespace ptp

extern "C" int ptp_residual_noalloc_dev(ptp_ctx* h, const double* U, double* R, double* norm);

// The context type is private to api.cpp; reach it through a small accessor.
namespace ptp {
Ctx* ctx_of(ptp_ctx* h);
int residual_grid(size_t total);
}

extern "C" int ptp_residual_noalloc_dev(ptp_ctx* h, const double* U, double* R, double* norm) {
    using namespace ptp;
    Ctx* cp = ctx_of(h);
    if (!cp) return PTP_EINVAL;
    Ctx& c = *cp;
    try {
        c.err.clear();
        if (!c.ready) throw Error(PTP_ESTATE, "call ptp_setup first");
        if (!U) throw Error(PTP_EINVAL, "ptp_residual_noalloc_dev: null U");
        PTP_CUDA(cudaSetDevice(c.device));
        const size_t flux = 2 * (size_t)c.n_iron * c.N;
        if (flux > kMaxFluxDoubles)
            throw Error(PTP_EINVAL,
                        "ptp_residual_noalloc_dev: the iron element fluxes need 2 * n_iron * N = " +
                            std::to_string(flux) + " doubles, above the fixed scratch of " +
                            std::to_string(kMaxFluxDoubles) + " (n_iron * N <= " +
                            std::to_string(kMaxFluxDoubles / 2) + "); use ptp_residual_dev");
        if ((size_t)residual_grid((size_t)c.n * c.N) > kPartialDoubles)
            throw Error(PTP_EINVAL, "ptp_residual_noalloc_dev: more residual blocks than partial-sum slots");
        double* base = static_cast<double*>(scratch_address(c.device));
        ResidualArgs a = residual_args(c, U, R);
        a.counter = reinterpret_cast<unsigned*>(base);
        a.partials = base + kCounterDoubles;
        a.Qx = base + kFluxOffset;
        a.Qy = a.Qx + (size_t)c.n_iron * c.N;
        a.status = nullptr;
        a.norm_out = norm;
        a.done = nullptr;
        a.check = 0;
        // the ticket counter must start at zero; the kernel resets it when done
        PTP_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(unsigned), c.stream));
        launch_residual_law(a, c.law_exp ? c.e_law.p : nullptr, c.stream);
        PTP_CUDA(cudaGetLastError());
        return PTP_OK;
    } catch (const Error& e) {
        c.err = e.what();
        return e.code;
    } catch (const std::exception& e) {
        c.err = e.what();
        return PTP_EINVAL;
    }
}
