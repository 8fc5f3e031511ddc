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
//
// In host code the array's name only stands for it; the kernel needs its
// device address, which cudaGetSymbolAddress returns for the CUDA context
// that is current.  The first call in a context looks that address up (the
// lookup may load the library's module, so make the first call before any
// stream capture) and keeps it for that context; a context created later on
// the same device (after cudaDeviceReset, say) gets its own lookup.
#include <cuda.h>

#include <map>
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

// The current context's identity, through the driver entry points the
// runtime hands out (no link against the driver library).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

struct DriverFns {
    CtxGetCurrentFn get_current = nullptr;
    CtxGetIdFn get_id = nullptr;
};

const DriverFns& driver_fns() {
    static DriverFns f = [] {
        DriverFns d;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            d.get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            d.get_id = reinterpret_cast<CtxGetIdFn>(p);
        return d;
    }();
    return f;
}

std::mutex g_mutex;
std::map<unsigned long long, void*> g_addr;   // device address of the array per CUDA context id

void* lookup_symbol() {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_residual_scratch);
    if (e != cudaSuccess || !p)
        throw Error(PTP_ECUDA, std::string("cudaGetSymbolAddress of the residual scratch failed: ") +
                                   cudaGetErrorString(e));
    return p;
}

// Device address of g_residual_scratch in the current context (the caller
// made the context's device current).
void* scratch_address() {
    const DriverFns& d = driver_fns();
    CUcontext cur = nullptr;
    unsigned long long id = 0;
    if (!d.get_current || !d.get_id || d.get_current(&cur) != CUDA_SUCCESS || !cur ||
        d.get_id(cur, &id) != CUDA_SUCCESS)
        return lookup_symbol();   // no context identity: look the address up on every call
    std::lock_guard<std::mutex> lock(g_mutex);
    auto it = g_addr.find(id);
    if (it != g_addr.end()) return it->second;
    void* p = lookup_symbol();
    g_addr[id] = p;
    return p;
}

}  // namespace

int residual_grid(size_t total);
}  // namespace ptp

extern "C" int ptp_residual_noalloc_dev(ptp_ctx* h, const double* U, double* R, double* norm) {
    using namespace ptp;
    return run_entry(h, [&](Ctx& c) {
        PTP_REQUIRE(U && (const void*)U != (const void*)R,
                    "ptp_residual_noalloc_dev: null U, or R is U (the residual would overwrite its input)");
        PTP_REQUIRE(!norm || ((const void*)norm != (const void*)U && (const void*)norm != (const void*)R),
                    "ptp_residual_noalloc_dev: norm aliases U or R");
        const size_t flux = 2 * (size_t)c.n_iron * c.N;
        if (flux > kMaxFluxDoubles)
            throw Error(PTP_EINVAL,
                        "ptp_residual_noalloc_dev: the iron element fluxes need 2 * n_iron * N = " +
                            std::to_string(flux) + " doubles, above the fixed scratch of " +
                            std::to_string(kMaxFluxDoubles) + " (n_iron * N <= " +
                            std::to_string(kMaxFluxDoubles / 2) + "); use ptp_residual_dev");
        if ((size_t)residual_grid((size_t)c.n * c.N) > kPartialDoubles)
            throw Error(PTP_EINVAL, "ptp_residual_noalloc_dev: more residual blocks than partial-sum slots");
        double* base = static_cast<double*>(scratch_address());
        ResidualArgs a = residual_args(c, U, R);
        a.counter = reinterpret_cast<unsigned*>(base);
        a.partials = base + kCounterDoubles;
        a.partials_cap = kPartialDoubles;
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
    });
}
