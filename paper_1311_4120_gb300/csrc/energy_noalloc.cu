// Energy reduction that allocates no memory: nlint_energy_noalloc.
//
// Some callers cannot allocate device memory at the point where they need the energy: code
// that runs while another framework owns every byte of the device through its own pool,
// a host thread that must not call cudaMalloc/cudaFree because those calls synchronise the
// device, or an embedded caller with a fixed memory budget decided up front.  The plan-based
// nlint_energy needs a plan, and creating a plan allocates.  This entry point needs neither:
// its only scratch is the file-scope device array below, reserved once when the library is
// loaded onto a device and held until the process exits.
//
// Scratch: one compensated (sum, correction) pair per CTA.  Each CTA reduces a fixed chunk of
// NOALLOC_CHUNK grid points, so the order of the additions, and hence the result, depends only
// on the inputs.  At most NOALLOC_MAX_PARTIALS CTAs fit, which bounds the grid at
// NOALLOC_MAX_POINTS points; larger grids are rejected with NLINT_EINVAL.
//
// Every call writes all the partial sums it later reads, so nothing has to be cleared between
// calls; the array keeps the last call's partial sums.  Calls share the one array, so two
// calls whose work overlaps on the GPU (different streams, or different host threads) race
// and give wrong energies: serialise them.
#include <cuda.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace nlint {

static constexpr int NOALLOC_THREADS = 256;
static constexpr int NOALLOC_PER_THREAD = 16;
static constexpr int64_t NOALLOC_CHUNK = (int64_t)NOALLOC_THREADS * NOALLOC_PER_THREAD;
static constexpr int NOALLOC_MAX_PARTIALS = 65536;  // 1 MiB of scratch
static constexpr int64_t NOALLOC_MAX_POINTS = NOALLOC_CHUNK * NOALLOC_MAX_PARTIALS;

static __device__ __align__(256) double2 g_noalloc_partials[NOALLOC_MAX_PARTIALS];

// Partial sums: CTA b reduces points [b*CHUNK, (b+1)*CHUNK) into partials[b].  Each thread
// sums its 16 products in FP64 (products of FP32 inputs are exact in FP64), then a fixed
// shuffle tree combines the threads with compensation.
template <typename T>
__global__ void __launch_bounds__(NOALLOC_THREADS) noalloc_partials_kernel(
    int64_t count, const T *__restrict__ u, const T *__restrict__ rho, double2 *__restrict__ partials) {
    __shared__ double sh[2 * 32];
    const int64_t base = (int64_t)blockIdx.x * NOALLOC_CHUNK;
    KSum acc;
    acc.init();
#pragma unroll
    for (int k = 0; k < NOALLOC_PER_THREAD; k++) {
        const int64_t i = base + (int64_t)k * NOALLOC_THREADS + threadIdx.x;
        if (i < count) acc.add((double)u[i] * (double)rho[i]);
    }
    KSum tot = ksum_block(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(tot.s, tot.c);
}

// One CTA folds the partials in a fixed order and writes scale * sum to E.
__global__ void __launch_bounds__(1024) noalloc_final_kernel(const double2 *__restrict__ partials,
                                                             int nparts, double scale,
                                                             double *__restrict__ E) {
    __shared__ double sh[2 * 32];
    KSum acc;
    acc.init();
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) acc.merge(partials[q].x, partials[q].y);
    KSum tot = ksum_block(acc, sh);
    if (threadIdx.x == 0) *E = scale * tot.value();
}

// Device address of the scratch array, looked up once per device and CUDA context with that
// device current.  In host code the array's name is only a host-side stand-in, never a device
// address.  The address belongs to the context the library's module was loaded into: after
// cudaDeviceReset, or under another context of the same device, the module is loaded again,
// possibly elsewhere, so the cache is keyed on the calling thread's current context (its
// process-unique ID from cuCtxGetId, reached through the runtime's driver entry points, so
// the library does not link the driver library) and the address is looked up again when that
// ID changes.
typedef int (*ctx_get_current_fn)(CUcontext *);
typedef int (*ctx_get_id_fn)(CUcontext, unsigned long long *);

static std::mutex g_noalloc_mu;
static double2 *g_noalloc_ptr[64];
static unsigned long long g_noalloc_ctx[64];  // context ID of the cached address, 0 = none
static ctx_get_current_fn g_ctx_get_current;
static ctx_get_id_fn g_ctx_get_id;

// Process-unique ID of the calling thread's current context, 0 when there is none yet.
static int current_context_id(unsigned long long *id) {
    *id = 0;
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return report_error(NLINT_ECUDA, "driver entry points cuCtxGetCurrent/cuCtxGetId unavailable");
        g_ctx_get_current = (ctx_get_current_fn)f1;
        g_ctx_get_id = (ctx_get_id_fn)f2;
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0) return report_error(NLINT_ECUDA, "cuCtxGetCurrent failed");
    if (ctx && g_ctx_get_id(ctx, id) != 0) return report_error(NLINT_ECUDA, "cuCtxGetId failed");
    return NLINT_OK;
}

static int noalloc_scratch(int dev, double2 **out) {
    if (dev < 0 || dev >= 64) return report_error(NLINT_EUNSUPPORTED, "device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    unsigned long long id = 0;
    int rc = current_context_id(&id);
    if (rc != NLINT_OK) return rc;
    if (id == 0 || g_noalloc_ctx[dev] != id) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess) {
            std::string m = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return report_error(NLINT_ECUDA, m.c_str());
        }
        if (id == 0) {  // the lookup made the device's primary context current
            rc = current_context_id(&id);
            if (rc != NLINT_OK) return rc;
        }
        g_noalloc_ptr[dev] = static_cast<double2 *>(ptr);
        g_noalloc_ctx[dev] = id;
    }
    *out = g_noalloc_ptr[dev];
    return NLINT_OK;
}

}  // namespace nlint

using namespace nlint;

extern "C" int nlint_energy_noalloc(int d, int64_t n, double L, int precision, const void *rho_dev,
                                    const void *u_dev, double lambda, double *E_dev, void *stream) {
    if (d != 2 && d != 3) return report_error(NLINT_EINVAL, "d must be 2 or 3");
    if (n < 1) return report_error(NLINT_EINVAL, "n must be positive");
    if (!(L > 0.0)) return report_error(NLINT_EINVAL, "L must be positive");
    if (precision != NLINT_FP32 && precision != NLINT_FP64)
        return report_error(NLINT_EINVAL, "precision must be NLINT_FP32 or NLINT_FP64");
    if (!rho_dev || !u_dev || !E_dev) return report_error(NLINT_EINVAL, "NULL rho, u or E");
    int64_t count = 1;
    for (int a = 0; a < d; a++) {
        if (count > NOALLOC_MAX_POINTS / n) {
            count = NOALLOC_MAX_POINTS + 1;
            break;
        }
        count *= n;
    }
    if (count > NOALLOC_MAX_POINTS)
        return report_error(NLINT_EINVAL,
                            "grid too large for nlint_energy_noalloc: at most 268435456 points "
                            "(65536 partial sums of 4096 points)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report_error(NLINT_ECUDA, cudaGetErrorString(e));
    double2 *partials = nullptr;
    int rc = noalloc_scratch(dev, &partials);
    if (rc != NLINT_OK) return rc;
    const int nblocks = (int)((count + NOALLOC_CHUNK - 1) / NOALLOC_CHUNK);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == NLINT_FP32)
        noalloc_partials_kernel<float><<<nblocks, NOALLOC_THREADS, 0, s>>>(
            count, (const float *)u_dev, (const float *)rho_dev, partials);
    else
        noalloc_partials_kernel<double><<<nblocks, NOALLOC_THREADS, 0, s>>>(
            count, (const double *)u_dev, (const double *)rho_dev, partials);
    const double h = L / (double)n;
    double hd = 1.0;
    for (int a = 0; a < d; a++) hd *= h;
    noalloc_final_kernel<<<1, 1024, 0, s>>>(partials, nblocks, 0.5 * lambda * hd, E_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(NLINT_ECUDA, cudaGetErrorString(e));
    return NLINT_OK;
}
