// Autotuner: picks the free parameters of a plan for a target accuracy and the fastest
// work decomposition, by measurement on the device, and caches the choice.
//
// Accuracy: the plan's spreading width w sets the NUFFT error (Section 2).  For a target
// relative L-inf error `tol`, the tuner evaluates a reference plan (same grid, nodes, cutoff
// and kernel; FP64 with the widest stencil) and candidate plans of the requested precision
// on a seeded probe density, and keeps the smallest w whose error is at most tol / 2.
// The probe is a sum of Gaussians whose widths range from two grid cells to an eighth of the
// box, so it has content up to the grid's Nyquist radius.
// Speed: for that w it times the bin shapes compiled for the plan's precision and dimension
// (the tile each interpolation / spreading CTA stages: 3D FP32 8^3, 8x16x16, 16^3; 3D FP64
// 8^3, 4x8x8; the shapes whose tile fits in shared memory at w), then, for the fastest shape,
// the subproblem sizes (nodes per CTA), and keeps the fastest pair.
// Cache: one JSON object per line in `cache_path` (or $NLINT_TUNE_CACHE), keyed by the plan's
// geometry, kernel, precision and tolerance; a hit skips all measurement.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

using namespace nlint;

namespace {

int tfail(int code, const char *msg) { return report_error(code, msg); }

// splitmix64: a seeded, platform-independent stream for the probe density
uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double unif(uint64_t &s) { return (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

std::vector<double> probe_density(int d, int64_t n, double L) {
    const double h = L / (double)n;
    uint64_t s = 0x1311412000000000ull + (uint64_t)n;
    const int G = 12;
    std::vector<double> c((size_t)G * 3), w(G), a(G);
    for (int g = 0; g < G; g++) {
        for (int k = 0; k < 3; k++) c[(size_t)g * 3 + k] = (unif(s) - 0.5) * 0.5 * L;
        w[g] = 2.0 * h * std::pow(L / (16.0 * h), (double)g / (G - 1));  // 2h .. L/8
        a[g] = 0.5 + unif(s);
    }
    int64_t count = 1;
    for (int k = 0; k < d; k++) count *= n;
    std::vector<double> rho((size_t)count, 0.0);
    for (int64_t i = 0; i < count; i++) {
        double x[3] = {0, 0, 0};
        int64_t r = i;
        for (int k = d - 1; k >= 0; k--) {  // C order: last index is x
            x[d - 1 - k] = -0.5 * L + h * (double)(r % n);
            r /= n;
        }
        double v = 0.0;
        for (int g = 0; g < G; g++) {
            double r2 = 0.0;
            for (int k = 0; k < d; k++) {
                const double t = x[k] - c[(size_t)g * 3 + k];
                r2 += t * t;
            }
            v += a[g] * std::exp(-r2 / (w[g] * w[g]));
        }
        rho[(size_t)i] = v;
    }
    return rho;
}

std::string cache_key(const nlint_params &p, double tol) {
    char buf[512];
    std::snprintf(buf, sizeof buf,
                  "d=%d n=%lld L=%.17g k=%d ax=%.17g,%.17g,%.17g ax2=%.17g,%.17g,%.17g al=%.17g "
                  "nodes=%lld,%lld,%lld P=%.17g s=%.17g prec=%d tol=%.3g",
                  p.d, (long long)p.n, p.L, p.kernel, p.axis[0], p.axis[1], p.axis[2], p.axis2[0],
                  p.axis2[1], p.axis2[2], p.alpha, (long long)p.n_r, (long long)p.n_theta,
                  (long long)p.n_phi, p.P, p.sigma, p.precision, tol);
    return buf;
}

bool cache_lookup(const char *path, const std::string &key, int &w, int &max_sub, int &bin_shape,
                  double &err) {
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[2048];
    bool hit = false;
    const std::string needle = "\"key\": \"" + key + "\"";
    while (std::fgets(line, sizeof line, f)) {
        if (!std::strstr(line, needle.c_str())) continue;
        const char *pw = std::strstr(line, "\"w\": ");
        const char *pm = std::strstr(line, "\"max_sub\": ");
        const char *pb = std::strstr(line, "\"bin_shape\": ");
        const char *pe = std::strstr(line, "\"err\": ");
        if (pw && pm && pb && pe) {  // lines without a bin shape are from an older tuner: a miss
            w = std::atoi(pw + 5);
            max_sub = std::atoi(pm + 11);
            bin_shape = std::atoi(pb + 13);
            err = std::atof(pe + 7);
            // the last matching line wins
            hit = w >= 2 && w <= NODE_MAXW && max_sub > 0 && bin_shape >= 1 && bin_shape <= NBIN_SHAPES;
        }
    }
    std::fclose(f);
    return hit;
}

void cache_store(const char *path, const std::string &key, int w, int max_sub, int bin_shape, double err,
                 double ms) {
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"key\": \"%s\", \"w\": %d, \"max_sub\": %d, \"bin_shape\": %d, \"err\": %.6g, "
                 "\"ms\": %.6g}\n",
                 key.c_str(), w, max_sub, bin_shape, err, ms);
    std::fclose(f);
}

struct Bufs {
    void *rho = nullptr, *u = nullptr;
    ~Bufs() {
        if (rho) cudaFree(rho);
        if (u) cudaFree(u);
    }
};

// u on the host (FP64) for plan p and the probe (uploaded in the plan's precision)
int eval_to_host(nlint_plan p, int prec, const std::vector<double> &rho, std::vector<double> &u,
                 cudaStream_t s) {
    const size_t cnt = rho.size(), es = prec == NLINT_FP32 ? 4 : 8;
    Bufs b;
    if (cudaMalloc(&b.rho, cnt * es) != cudaSuccess || cudaMalloc(&b.u, cnt * es) != cudaSuccess)
        return tfail(NLINT_ENOMEM, "autotune: device allocation failed");
    if (prec == NLINT_FP32) {
        std::vector<float> r(rho.begin(), rho.end());
        if (cudaMemcpy(b.rho, r.data(), cnt * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return tfail(NLINT_ECUDA, "autotune: copy failed");
    } else if (cudaMemcpy(b.rho, rho.data(), cnt * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        return tfail(NLINT_ECUDA, "autotune: copy failed");
    }
    int rc = nlint_eval(p, b.rho, b.u, s);
    if (rc) return rc;
    u.resize(cnt);
    if (prec == NLINT_FP32) {
        std::vector<float> h(cnt);
        if (cudaMemcpyAsync(h.data(), b.u, cnt * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return tfail(NLINT_ECUDA, "autotune: copy failed");
        for (size_t i = 0; i < cnt; i++) u[i] = h[i];
    } else if (cudaMemcpyAsync(u.data(), b.u, cnt * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
               cudaStreamSynchronize(s) != cudaSuccess) {
        return tfail(NLINT_ECUDA, "autotune: copy failed");
    }
    return NLINT_OK;
}

double rel_linf(const std::vector<double> &a, const std::vector<double> &b) {
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < a.size(); i++) {
        num = std::fmax(num, std::fabs(a[i] - b[i]));
        den = std::fmax(den, std::fabs(b[i]));
    }
    return den > 0.0 ? num / den : num;
}

// median time (ms) of `reps` evaluations of plan p on device buffers
int time_plan(nlint_plan p, int prec, const std::vector<double> &rho, int reps, cudaStream_t s, double &ms) {
    const size_t cnt = rho.size(), es = prec == NLINT_FP32 ? 4 : 8;
    Bufs b;
    if (cudaMalloc(&b.rho, cnt * es) != cudaSuccess || cudaMalloc(&b.u, cnt * es) != cudaSuccess)
        return tfail(NLINT_ENOMEM, "autotune: device allocation failed");
    cudaError_t ce;
    if (prec == NLINT_FP32) {  // time on the probe itself (a zero density would skip work)
        std::vector<float> r(rho.begin(), rho.end());
        ce = cudaMemcpy(b.rho, r.data(), cnt * 4, cudaMemcpyHostToDevice);
    } else {
        ce = cudaMemcpy(b.rho, rho.data(), cnt * 8, cudaMemcpyHostToDevice);
    }
    if (ce != cudaSuccess) return tfail(NLINT_ECUDA, "autotune: copy failed");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = nlint_eval(p, b.rho, b.u, s);  // warm-up
    std::vector<float> t;
    for (int r = 0; r < reps && rc == NLINT_OK; r++) {
        cudaEventRecord(e0, s);
        rc = nlint_eval(p, b.rho, b.u, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    std::sort(t.begin(), t.end());
    ms = t.empty() ? 0.0 : t[t.size() / 2];
    return NLINT_OK;
}

}  // namespace

extern "C" int nlint_autotune(const nlint_params *in, double tol, const char *cache_path,
                              nlint_params *out, nlint_tune_report *rep) {
    if (!in || !out) return tfail(NLINT_EINVAL, "NULL argument");
    if (!(tol > 0.0) || !(tol < 1.0)) return tfail(NLINT_EINVAL, "tol must be in (0, 1)");
    nlint_params p = *in;
    if (p.precision != NLINT_FP32 && p.precision != NLINT_FP64)
        p.precision = tol >= 1e-7 ? NLINT_FP32 : NLINT_FP64;
    if (!cache_path) cache_path = std::getenv("NLINT_TUNE_CACHE");
    const std::string key = cache_key(p, tol);
    int w = 0, max_sub = 0, bshape = 0;
    double err = 0.0, ms = 0.0;
    if (cache_lookup(cache_path, key, w, max_sub, bshape, err)) {
        p.w = w;
        p.max_sub = max_sub;
        p.bin_shape = bshape;
        *out = p;
        if (rep) *rep = nlint_tune_report{w, max_sub, err, 0.0, 1, bshape};
        return NLINT_OK;
    }
    if (p.device >= 0 && cudaSetDevice(p.device) != cudaSuccess)
        return tfail(NLINT_ECUDA, "autotune: cudaSetDevice failed");
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        return tfail(NLINT_ECUDA, "autotune: stream creation failed");
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{s};
    const std::vector<double> rho = probe_density(p.d, p.n, p.L);

    // reference: FP64, widest stencil
    nlint_params rp = p;
    rp.precision = NLINT_FP64;
    rp.w = NODE_MAXW;
    rp.eps = 1e-14;
    nlint_plan ref = nullptr;
    int rc = nlint_plan_create_ex(&rp, &ref);
    if (rc) return rc;
    std::vector<double> uref;
    rc = eval_to_host(ref, NLINT_FP64, rho, uref, s);
    nlint_plan_destroy(ref);
    if (rc) return rc;

    // smallest width whose error is at most tol / 2
    int best_w = -1;
    double best_err = 0.0;
    std::string tried;
    for (int cw = 2; cw <= NODE_MAXW && best_w < 0; cw++) {
        nlint_params cp = p;
        cp.w = cw;
        nlint_plan pl = nullptr;
        if (nlint_plan_create_ex(&cp, &pl) != NLINT_OK) continue;  // e.g. grid too small for w
        std::vector<double> u;
        rc = eval_to_host(pl, p.precision, rho, u, s);
        nlint_plan_destroy(pl);
        if (rc) return rc;
        const double e = rel_linf(u, uref);
        char b[48];
        std::snprintf(b, sizeof b, " w=%d:%.2e", cw, e);
        tried += b;
        if (e <= 0.5 * tol) {
            best_w = cw;
            best_err = e;
        }
    }
    if (best_w < 0) {
        const std::string m = "autotune: no stencil width reaches the tolerance (errors" + tried + ")";
        return tfail(NLINT_EUNSUPPORTED, m.c_str());
    }

    // fastest bin shape at that width (default subproblem size), then the fastest subproblem size
    // for that shape; a shape whose tile does not fit at this width is skipped
    auto time_candidate = [&](int bs, int cs, double &t) -> int {
        nlint_params cp = p;
        cp.w = best_w;
        cp.max_sub = cs;
        cp.bin_shape = bs;
        nlint_plan pl = nullptr;
        const int crc = nlint_plan_create_ex(&cp, &pl);
        if (crc == NLINT_EUNSUPPORTED) return crc;
        if (crc) return crc;
        const int trc = time_plan(pl, p.precision, rho, 5, s, t);
        nlint_plan_destroy(pl);
        return trc;
    };
    const bool f64 = p.precision == NLINT_FP64;
    int best_bs = 0, best_sub = 0;
    double best_ms = 1e30;
    for (int bs = 1; bs <= NBIN_SHAPES; bs++) {
        if (!bin_shape_built(f64, p.d, bs)) continue;
        double t = 0.0;
        rc = time_candidate(bs, 0, t);
        if (rc == NLINT_EUNSUPPORTED) continue;
        if (rc) return rc;
        if (t < best_ms) {
            best_ms = t;
            best_bs = bs;
        }
    }
    if (best_bs == 0) return tfail(NLINT_EUNSUPPORTED, "autotune: no bin shape fits at this width");
    const int cands[] = {256, 512, 1024, 2048};
    best_ms = 1e30;
    for (int cs : cands) {
        double t = 0.0;
        rc = time_candidate(best_bs, cs, t);
        if (rc) return rc;
        if (t < best_ms) {
            best_ms = t;
            best_sub = cs;
        }
    }
    p.w = best_w;
    p.max_sub = best_sub;
    p.bin_shape = best_bs;
    cache_store(cache_path, key, best_w, best_sub, best_bs, best_err, best_ms);
    *out = p;
    if (rep) *rep = nlint_tune_report{best_w, best_sub, best_err, best_ms, 0, best_bs};
    return NLINT_OK;
}
