// klecgc_reference_noalloc: the sequential fine solution of klecgc_reference
// computed without allocating device memory.
//
// Some callers cannot allocate device memory at the moment they need a
// result: code that runs inside another framework's memory budget (a caching
// allocator that owns all free device memory), real-time or embedded hosts
// that forbid allocation after start-up, and callbacks that must not
// synchronize the device (cudaMalloc/cudaFree may do so).  This entry point
// takes its working memory from one file-scope device array instead.  The
// array (kScratchBytes) is part of the library image: every GPU that loads
// the library holds it until the process exits.
#include <mutex>
#include <string>

#include "../../include/klecgc.h"
#include "common.cuh"
#include "ptr_rule.h"

namespace klecgc {

namespace {

constexpr size_t kScratchBytes = 32u << 20;                  // 32 MiB
constexpr size_t kScratchDoubles = kScratchBytes / sizeof(double);

// Shared by every call: it keeps the previous call's contents, and calls whose
// GPU work overlaps (e.g. on two streams at once) race on it.
static __device__ __align__(256) double g_scratch[kScratchDoubles];

// Device address of g_scratch per CUDA device.  In host code the name
// g_scratch is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

cudaError_t scratch_address(int dev, double** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// true for device memory of device `dev` and for managed memory
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return device_array_usable((int)a.type, a.device, dev);
}

// N*J sequential backward-Euler steps per sample (one thread per sample), the
// state in scratch[nx][S]; writes U[s][n][i] (the caller's layout) directly.
__global__ void __launch_bounds__(64) k_fine_sequential_user(
    int64_t S, int N, int nx, int J, double dtf, const double* __restrict__ u0,
    const FineCoef64* __restrict__ fc, double* __restrict__ state, double* __restrict__ U) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= S) return;
    const FineCoef64* c = fc + s * (nx + 1);
    for (int i = 0; i < nx; ++i) state[(int64_t)i * S + s] = u0[i];
    for (int n = 0; n < N; ++n) {
        for (int j = 0; j < J; ++j) {
            double y = 0.0;
            for (int i = 0; i < nx; ++i) {
                double* p = state + (int64_t)i * S + s;
                y = fma(-c[i].l, y, *p + dtf);
                *p = y;
            }
            double x = 0.0;
            for (int i = nx - 1; i >= 0; --i) {
                double* p = state + (int64_t)i * S + s;
                x = fma(c[i + 1].wd, x, *p) * c[i].dinv;
                *p = x;
            }
        }
        double* Un = U + (s * N + n) * (int64_t)nx;
        for (int i = 0; i < nx; ++i) Un[i] = state[(int64_t)i * S + s];
    }
}

klecgc_status fail_na(klecgc_status s, const std::string& m) {
    set_error(m);
    return s;
}

}  // namespace
}  // namespace klecgc

using namespace klecgc;

extern "C" klecgc_status klecgc_reference_noalloc(klecgc_ctx* ctx, const double* xi, int64_t S,
                                                  int32_t N, int32_t J, double* U_out,
                                                  void* stream) {
    set_error("");
    CtxView cv;
    if (!ctx || !ctx_view(ctx, &cv) || S < 0 || N < 1 || J < 1)
        return fail_na(KLECGC_E_INVALID_ARG, "bad argument");
    if (cv.dim != 1 || cv.reaction_kind != 0)
        return fail_na(KLECGC_E_UNSUPPORTED,
                       "the allocation-free entry point takes the linear 1D problem only");
    if (S == 0) return KLECGC_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != cv.device || dev >= kMaxDevices)
        return fail_na(KLECGC_E_INVALID_ARG, "the context's device must be current");
    if (!on_device(xi, cv.device) || !on_device(U_out, cv.device))
        return fail_na(KLECGC_E_INVALID_ARG,
                       "xi and U_out must be device (or managed) arrays of the context's device");
    // scratch: fine factors [S][nx+1] (4 doubles each), field a [S][nx+1], state [nx][S]:
    // S (6 nx + 5) doubles.  Compared as S against the largest admissible
    // count, so that no product can wrap.
    const int64_t nf = cv.nx + 1;
    const int64_t per_sample = 5 * nf + cv.nx;
    const int64_t s_max = (int64_t)(kScratchDoubles / (size_t)per_sample);
    if (S > s_max)
        return fail_na(KLECGC_E_INVALID_ARG,
                       "S = " + std::to_string(S) + " at nx = " + std::to_string(cv.nx) +
                           " exceeds the static scratch: S * (6 nx + 5) must be at most " +
                           std::to_string(kScratchDoubles) + " doubles (32 MiB), S at most " +
                           std::to_string(s_max));
    double* base = nullptr;
    cudaError_t e = scratch_address(dev, &base);
    if (e != cudaSuccess)
        return fail_na(KLECGC_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    FineCoef64* fc = reinterpret_cast<FineCoef64*>(base);         // 256-byte aligned
    double* a = base + 4 * S * nf;
    double* state = a + S * nf;
    cudaStream_t st = (cudaStream_t)stream;
    const double dt = cv.T / N / J;
    // every scratch word that is read is written first in this call: nothing
    // has to start at zero
    launch_field(xi, S, cv.M, cv.basis, (int)nf, a, st);
    launch_fine_factors(a, S, cv.nx, cv.h, dt, cv.reaction, fc, nullptr, st);
    k_fine_sequential_user<<<(unsigned)((S + 63) / 64), 64, 0, st>>>(S, N, cv.nx, J,
                                                                    dt * cv.forcing, cv.u0, fc,
                                                                    state, U_out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_na(KLECGC_E_CUDA, cudaGetErrorString(e));
    return KLECGC_OK;
}
