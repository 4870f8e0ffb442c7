// Batched evaluation: many densities, each with its own plan (grid size, kernel, precision),
// evaluated by one CUDA graph.
//
// The graph is captured once per set of argument pointers: a fork from an origin stream into
// S branch streams, each branch running its share of the plans' full evaluations (type-2 NUFFT,
// multiply, type-1 NUFFT, energy) back to back, and a join.  Plans are dealt to branches by
// longest-processing-time-first on a cost model (grid points plus node work), so the branches
// finish together; inside the graph the branches run concurrently and fill the GPU with the
// small grids' kernels that would each leave most SMs idle.  A replay is one
// cudaGraphLaunch on the caller's stream.  This is the batched form of Algorithm 1 (Section
// 3.2) applied to independent densities; the paper evaluates one density at a time.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"

using namespace nlint;

struct nlint_batch_s {
    std::vector<nlint_plan> plans;
    int device = 0;
    std::vector<cudaStream_t> branch;
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    std::vector<std::vector<int>> deal;  // plan indices per branch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // arguments the current graph was captured with
    std::vector<const void *> key_rho;
    std::vector<void *> key_u;
    double key_lambda = 0.0;
    double *key_E = nullptr;
    int64_t kernels = 0;  // kernels per replay
};

static int bfail(int code, const char *msg) { return report_error(code, msg); }
static int bcuda(cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return report_error(NLINT_ECUDA, m.c_str());
}
#define BCK(call)                                             \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return bcuda(e_, #call);       \
    } while (0)

static void batch_free(nlint_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaStream_t s : b->branch) cudaStreamDestroy(s);
    if (b->origin) cudaStreamDestroy(b->origin);
}

extern "C" {

int nlint_batch_create(int count, const nlint_plan *plans, int branches, nlint_batch *out) {
    if (!out) return bfail(NLINT_EINVAL, "NULL output");
    *out = nullptr;
    if (count <= 0 || !plans) return bfail(NLINT_EINVAL, "count must be positive and plans non-NULL");
    nlint_batch_s *b = new (std::nothrow) nlint_batch_s();
    if (!b) return bfail(NLINT_ENOMEM, "host allocation failed");
    std::vector<double> cost(count);
    int dev = -1;
    for (int i = 0; i < count; i++) {
        nlint_info inf;
        if (!plans[i] || nlint_plan_info(plans[i], &inf) != NLINT_OK) {
            delete b;
            return bfail(NLINT_EINVAL, "invalid plan in the batch");
        }
        // a plan owns one set of workspaces: two of its evaluations on different branches of
        // the graph would run at the same time on them and corrupt both results
        for (int j = 0; j < i; j++)
            if (plans[j] == plans[i]) {
                delete b;
                return bfail(NLINT_EINVAL, "a plan appears more than once in the batch");
            }
        const int pdev = inf.device;
        if (dev < 0) dev = pdev;
        if (pdev != dev) {
            delete b;
            return bfail(NLINT_EINVAL, "all plans of a batch must be on one device");
        }
        double pts = 1.0;
        for (int a = 0; a < inf.d; a++) pts *= (double)inf.n_fine;
        // cost model: oversampled-grid traffic plus node work (w^d per node), in grid-point units
        // (a plan with a precomputed Toeplitz kernel runs FFT passes only)
        cost[i] = 3.0 * pts + (inf.toeplitz ? 0.0
                                            : (double)inf.n_half_nodes * std::pow((double)inf.w, inf.d) /
                                                  8.0 * (inf.precision == NLINT_FP64 ? 16.0 : 1.0));
        b->plans.push_back(plans[i]);
    }
    b->device = dev;
    int rc = NLINT_OK;
    if (cudaSetDevice(dev) != cudaSuccess) rc = bfail(NLINT_ECUDA, "cudaSetDevice failed");
    const int S = std::max(1, std::min(branches > 0 ? branches : 16, count));
    if (rc == NLINT_OK) {
        b->deal.assign(S, {});
        std::vector<int> ord(count);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        std::vector<double> load(S, 0.0);
        for (int i : ord) {
            const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            b->deal[k].push_back(i);
            load[k] += cost[i];
        }
        cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (int k = 0; k < S && e == cudaSuccess; k++) {
            cudaStream_t s;
            cudaEvent_t ev;
            e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e == cudaSuccess) b->branch.push_back(s);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) b->join.push_back(ev);
        }
        if (e != cudaSuccess) rc = bcuda(e, "creating the batch's streams");
    }
    if (rc != NLINT_OK) {
        batch_free(b);
        delete b;
        return rc;
    }
    *out = b;
    return NLINT_OK;
}

static int batch_capture(nlint_batch_s *b, const void *const *rho, void *const *u, double lambda,
                         double *E_dev) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    int64_t before = 0, after = 0;
    for (nlint_plan p : b->plans) {
        int64_t c = 0;
        nlint_launch_count(p, &c);
        before += c;
    }
    BCK(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed));
    int rc = NLINT_OK;
    cudaError_t e = cudaEventRecord(b->fork, b->origin);
    for (size_t k = 0; k < b->branch.size() && e == cudaSuccess; k++)
        e = cudaStreamWaitEvent(b->branch[k], b->fork, 0);
    for (size_t k = 0; k < b->branch.size() && e == cudaSuccess && rc == NLINT_OK; k++) {
        for (int i : b->deal[k]) {
            nlint_info inf;
            rc = nlint_plan_info(b->plans[i], &inf);
            if (rc != NLINT_OK) break;
            double *Ei = E_dev ? E_dev + i : nullptr;
            rc = inf.toeplitz ? nlint_eval_toeplitz(b->plans[i], rho[i], u[i], lambda, Ei, (void *)b->branch[k])
                              : nlint_eval_energy(b->plans[i], rho[i], u[i], lambda, Ei, (void *)b->branch[k]);
            if (rc != NLINT_OK) break;
        }
        if (rc == NLINT_OK) e = cudaEventRecord(b->join[k], b->branch[k]);
        if (e == cudaSuccess && rc == NLINT_OK) e = cudaStreamWaitEvent(b->origin, b->join[k], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->origin, &g);
    if (rc != NLINT_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(e, "recording the batch graph");
    }
    if (ee != cudaSuccess) return bcuda(ee, "cudaStreamEndCapture");
    b->graph = g;
    BCK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    for (nlint_plan p : b->plans) {
        int64_t c = 0;
        nlint_launch_count(p, &c);
        after += c;
    }
    b->kernels = after - before;
    b->key_rho.assign(rho, rho + b->plans.size());
    b->key_u.assign(u, u + b->plans.size());
    b->key_lambda = lambda;
    b->key_E = E_dev;
    return NLINT_OK;
}

int nlint_batch_eval(nlint_batch b, const void *const *rho, void *const *u, double lambda,
                     double *E_dev, void *stream) {
    if (!b) return bfail(NLINT_EINVAL, "batch is NULL");
    if (!rho || !u) return bfail(NLINT_EINVAL, "NULL rho or u array");
    const size_t c = b->plans.size();
    for (size_t i = 0; i < c; i++)
        if (!rho[i] || !u[i]) return bfail(NLINT_EINVAL, "NULL rho or u pointer in the batch");
    BCK(cudaSetDevice(b->device));
    const bool same = b->exec && b->key_lambda == lambda && b->key_E == E_dev &&
                      std::equal(b->key_rho.begin(), b->key_rho.end(), rho) &&
                      std::equal(b->key_u.begin(), b->key_u.end(), u);
    if (!same) {
        const int rc = batch_capture(b, rho, u, lambda, E_dev);
        if (rc != NLINT_OK) return rc;
    }
    BCK(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return NLINT_OK;
}

int nlint_batch_info(nlint_batch b, int *count, int *branches, int64_t *kernels_per_eval) {
    if (!b) return bfail(NLINT_EINVAL, "batch is NULL");
    if (count) *count = (int)b->plans.size();
    if (branches) *branches = (int)b->branch.size();
    if (kernels_per_eval) *kernels_per_eval = b->kernels;
    return NLINT_OK;
}

void nlint_batch_destroy(nlint_batch b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    batch_free(b);
    delete b;
}

}  // extern "C"
