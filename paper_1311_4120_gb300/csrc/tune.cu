// Autotuner: picks the free parameters of a plan for a target accuracy and the fastest
// work decomposition, by measurement on the device, and caches the choice.
//
// Accuracy: the plan's spreading width w sets the NUFFT error (Section 2).  For a target
// relative L-inf error `tol`, the tuner evaluates a reference plan (same grid, nodes, cutoff
// and kernel; FP64 with the widest stencil) and candidate plans of the requested precision
// on a seeded probe density, and keeps the smallest w whose error is at most tol / 2.
// The probe is a sum of Gaussians whose widths range from two grid cells to an eighth of the
// box, so it has content up to the grid's Nyquist radius.
// Speed: for that w and the next one (also within the tolerance, and sometimes faster: the
// node kernels' lane layout depends on w) it times the bin shapes compiled for the plan's
// precision and dimension (the tile each interpolation / spreading CTA stages: 3D FP32 8^3,
// 8x16x16, 16^3; 3D FP64 8^3, 4x8x8; the shapes whose tile fits in shared memory at w), then,
// for the fastest width and shape, the subproblem sizes (nodes per CTA), and keeps the fastest;
// then (FP32) the FFT pass schedules, one pass class at a time (coordinate descent over the
// four bits of nlint_params.fft_sched), each kept when the evaluation's FFT stages (timed by the
// plan's stage events) measured at least 1 % faster.
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
                  double &err, int &w_alt, double &err_alt, int &fft_sched) {
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
        const char *pa = std::strstr(line, "\"w_alt\": ");
        const char *pea = std::strstr(line, "\"err_alt\": ");
        const char *pfs = std::strstr(line, "\"fft_sched\": ");
        if (pw && pm && pb && pe) {  // lines without a bin shape are from an older tuner: a miss
            w = std::atoi(pw + 5);
            max_sub = std::atoi(pm + 11);
            bin_shape = std::atoi(pb + 13);
            err = std::atof(pe + 7);
            w_alt = (pa && pea) ? std::atoi(pa + 9) : 0;
            err_alt = (pa && pea) ? std::atof(pea + 11) : 0.0;
            fft_sched = pfs ? std::atoi(pfs + 13) : 0;
            // the last matching line wins
            hit = w >= 2 && w <= NODE_MAXW && max_sub > 0 && bin_shape >= 1 && bin_shape <= NBIN_SHAPES;
        }
    }
    std::fclose(f);
    return hit;
}

void cache_store(const char *path, const std::string &key, int w, int max_sub, int bin_shape, double err,
                 double ms, int w_alt, double err_alt, int fft_sched) {
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"key\": \"%s\", \"w\": %d, \"max_sub\": %d, \"bin_shape\": %d, \"err\": %.6g, "
                 "\"ms\": %.6g, \"w_alt\": %d, \"err_alt\": %.6g, \"fft_sched\": %d}\n",
                 key.c_str(), w, max_sub, bin_shape, err, ms, w_alt, err_alt, fft_sched);
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

// median of `reps` evaluations of plan p of the summed times of its FFT stages (the stage events
// of nlint_stage_times whose names name an FFT pass): the part of an evaluation that the FFT
// pass schedules change, without the node kernels' larger share and its variation
int time_fft_stages(nlint_plan p, int prec, const std::vector<double> &rho, int reps, cudaStream_t s,
                    double &ms) {
    const size_t cnt = rho.size(), es = prec == NLINT_FP32 ? 4 : 8;
    Bufs b;
    if (cudaMalloc(&b.rho, cnt * es) != cudaSuccess || cudaMalloc(&b.u, cnt * es) != cudaSuccess)
        return tfail(NLINT_ENOMEM, "autotune: device allocation failed");
    cudaError_t ce;
    if (prec == NLINT_FP32) {
        std::vector<float> r(rho.begin(), rho.end());
        ce = cudaMemcpy(b.rho, r.data(), cnt * 4, cudaMemcpyHostToDevice);
    } else {
        ce = cudaMemcpy(b.rho, rho.data(), cnt * 8, cudaMemcpyHostToDevice);
    }
    if (ce != cudaSuccess) return tfail(NLINT_ECUDA, "autotune: copy failed");
    int rc = nlint_eval(p, b.rho, b.u, s);  // warm-up
    if (rc) return rc;
    if ((rc = nlint_set_stage_timing(p, 1))) return rc;
    std::vector<double> t;
    for (int r = 0; r < reps && rc == NLINT_OK; r++) {
        rc = nlint_eval(p, b.rho, b.u, s);
        float st[32];
        const char *nm[32];
        int k = 0;
        if (rc == NLINT_OK) rc = nlint_stage_times(p, st, nm, 32, &k);
        double sum = 0.0;
        for (int i = 0; i < k && rc == NLINT_OK; i++)
            if (std::strstr(nm[i], "fft") || std::strstr(nm[i], "dual")) sum += st[i];
        t.push_back(sum);
    }
    nlint_set_stage_timing(p, 0);
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
    int w = 0, max_sub = 0, bshape = 0, walt = 0, fsched = 0;
    double err = 0.0, ealt = 0.0;
    if (cache_lookup(cache_path, key, w, max_sub, bshape, err, walt, ealt, fsched)) {
        p.w = w;
        p.max_sub = max_sub;
        p.bin_shape = bshape;
        p.fft_sched = fsched;
        *out = p;
        if (rep) *rep = nlint_tune_report{w, max_sub, err, 0.0, 1, bshape, walt, ealt, fsched};
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

    // fastest (width, bin shape) at the default subproblem size, over the smallest qualifying
    // width and the next one (which also meets the tolerance, with a smaller error, and can be
    // faster: the lane layout of the node kernels depends on w), then the fastest subproblem size
    // for that pair; a shape whose tile does not fit at a width is skipped
    auto time_candidate = [&](int cw, int bs, int cs, double &t, int fs = 0) -> int {
        nlint_params cp = p;
        cp.w = cw;
        cp.max_sub = cs;
        cp.bin_shape = bs;
        cp.fft_sched = fs;
        nlint_plan pl = nullptr;
        const int crc = nlint_plan_create_ex(&cp, &pl);
        if (crc == NLINT_EUNSUPPORTED) return crc;
        if (crc) return crc;
        const int trc = time_plan(pl, p.precision, rho, 5, s, t);
        nlint_plan_destroy(pl);
        return trc;
    };
    const bool f64 = p.precision == NLINT_FP64;
    int best_bs = 0, best_sub = 0, fast_w = best_w, alt_w = 0;
    double best_ms = 1e30;
    for (int cw = best_w; cw <= std::min(best_w + 1, (int)NODE_MAXW); cw++) {
        bool timed = false;
        for (int bs = 1; bs <= NBIN_SHAPES; bs++) {
            if (!bin_shape_built(f64, p.d, bs)) continue;
            double t = 0.0;
            rc = time_candidate(cw, bs, 0, t);
            if (rc == NLINT_EUNSUPPORTED) continue;
            if (rc) return rc;
            timed = true;
            if (t < best_ms) {
                best_ms = t;
                best_bs = bs;
                fast_w = cw;
            }
        }
        if (timed && cw > best_w) alt_w = cw;  // the next width ran: the choice or the alternative
    }
    if (best_bs == 0) return tfail(NLINT_EUNSUPPORTED, "autotune: no bin shape fits at this width");
    // the error of the wider width, measured as for the smallest one: it is either the choice
    // (the faster one) or the alternative, which must then meet the tolerance too
    double alt_err = 0.0;
    if (alt_w) {
        nlint_params cp = p;
        cp.w = alt_w;
        nlint_plan pl = nullptr;
        rc = nlint_plan_create_ex(&cp, &pl);
        if (rc) return rc;
        std::vector<double> u;
        rc = eval_to_host(pl, p.precision, rho, u, s);
        nlint_plan_destroy(pl);
        if (rc) return rc;
        const double e = rel_linf(u, uref);
        if (fast_w == alt_w) {
            alt_w = best_w;
            alt_err = best_err;
            best_w = fast_w;
            best_err = e;
        } else if (e <= 0.5 * tol) {
            alt_err = e;
        } else {
            alt_w = 0;
        }
    }
    const int cands[] = {256, 512, 1024, 2048};
    best_ms = 1e30;
    for (int cs : cands) {
        double t = 0.0;
        rc = time_candidate(best_w, best_bs, cs, t);
        if (rc) return rc;
        if (t < best_ms) {
            best_ms = t;
            best_sub = cs;
        }
    }
    // FFT pass schedules (FP32): one pass class at a time, kept when the evaluation's FFT stages
    // measured at least 1 % faster (their own stage events: the schedules change nothing else)
    int best_fs = 0;
    if (!f64) {
        auto fft_ms = [&](int fs, double &t) -> int {
            nlint_params cp = p;
            cp.w = best_w;
            cp.max_sub = best_sub;
            cp.bin_shape = best_bs;
            cp.fft_sched = fs;
            nlint_plan pl = nullptr;
            const int crc = nlint_plan_create_ex(&cp, &pl);
            if (crc) return crc;
            const int trc = time_fft_stages(pl, p.precision, rho, 9, s, t);
            nlint_plan_destroy(pl);
            return trc;
        };
        double base = 0.0;
        rc = fft_ms(0, base);
        if (rc) return rc;
        for (int bit = 0; bit < 4; bit++) {
            double t = 0.0;
            rc = fft_ms(best_fs | (1 << bit), t);
            if (rc) return rc;
            if (t < 0.99 * base) {
                base = t;
                best_fs |= 1 << bit;
            }
        }
        if (best_fs) {  // the evaluation time of the final choice
            rc = time_candidate(best_w, best_bs, best_sub, best_ms, best_fs);
            if (rc) return rc;
        }
    }
    p.w = best_w;
    p.max_sub = best_sub;
    p.bin_shape = best_bs;
    p.fft_sched = best_fs;
    cache_store(cache_path, key, best_w, best_sub, best_bs, best_err, best_ms, alt_w, alt_err, best_fs);
    *out = p;
    if (rep) *rep = nlint_tune_report{best_w, best_sub, best_err, best_ms, 0, best_bs, alt_w, alt_err, best_fs};
    return NLINT_OK;
}

namespace {

// The members' plans, batch and buffers for one timed decomposition; everything is released
// by the destructor.
struct BatchTrial {
    std::vector<nlint_plan> plans;
    std::vector<void *> rho, u;
    nlint_batch batch = nullptr;
    ~BatchTrial() {
        if (batch) nlint_batch_destroy(batch);
        for (nlint_plan p : plans) nlint_plan_destroy(p);
        for (void *q : rho) cudaFree(q);
        for (void *q : u) cudaFree(q);
    }
};

// median time (ms) of `reps` evaluations of the batch built from `prm` (one plan per member),
// on each member's probe density
int time_batch(const std::vector<nlint_params> &prm, int branches, int reps, cudaStream_t s, double &ms) {
    BatchTrial t;
    const int count = (int)prm.size();
    for (int i = 0; i < count; i++) {
        nlint_plan pl = nullptr;
        const int rc = nlint_plan_create_ex(&prm[(size_t)i], &pl);
        if (rc) return rc;
        t.plans.push_back(pl);
        int64_t cnt = 1;
        for (int k = 0; k < prm[(size_t)i].d; k++) cnt *= prm[(size_t)i].n;
        const size_t es = prm[(size_t)i].precision == NLINT_FP32 ? 4 : 8;
        void *r = nullptr, *u = nullptr;
        if (cudaMalloc(&r, (size_t)cnt * es) != cudaSuccess) return tfail(NLINT_ENOMEM, "autotune: device allocation failed");
        t.rho.push_back(r);
        if (cudaMalloc(&u, (size_t)cnt * es) != cudaSuccess) return tfail(NLINT_ENOMEM, "autotune: device allocation failed");
        t.u.push_back(u);
        const std::vector<double> rho = probe_density(prm[(size_t)i].d, prm[(size_t)i].n, prm[(size_t)i].L);
        cudaError_t ce;
        if (es == 4) {
            std::vector<float> f(rho.begin(), rho.end());
            ce = cudaMemcpy(r, f.data(), (size_t)cnt * 4, cudaMemcpyHostToDevice);
        } else {
            ce = cudaMemcpy(r, rho.data(), (size_t)cnt * 8, cudaMemcpyHostToDevice);
        }
        if (ce != cudaSuccess) return tfail(NLINT_ECUDA, "autotune: copy failed");
    }
    int rc = nlint_batch_create(count, t.plans.data(), branches, &t.batch);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> ts;
    for (int r = 0; r < reps + 2 && rc == NLINT_OK; r++) {  // two warm-up evaluations (the first captures)
        cudaEventRecord(e0, s);
        rc = nlint_batch_eval(t.batch, t.rho.data(), t.u.data(), 1.0, nullptr, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess && rc == NLINT_OK)
            rc = tfail(NLINT_ECUDA, "autotune: batch evaluation failed");
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        if (r >= 2) ts.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    std::sort(ts.begin(), ts.end());
    ms = ts.empty() ? 0.0 : ts[ts.size() / 2];
    return NLINT_OK;
}

}  // namespace

extern "C" int nlint_autotune_batch(int count, const nlint_params *in, double tol, const char *cache_path,
                                    int branches, nlint_params *out, nlint_tune_report *member_reps,
                                    nlint_batch_tune_report *rep) {
    if (count < 1 || !in || !out) return tfail(NLINT_EINVAL, "autotune_batch: count >= 1 and non-NULL in/out required");
    for (int i = 1; i < count; i++)
        if (in[i].device != in[0].device)
            return tfail(NLINT_EINVAL, "autotune_batch: members on different devices");
    if (!cache_path) cache_path = std::getenv("NLINT_TUNE_CACHE");
    // one tuning per class: the geometry, kernel, precision and tolerance of the cache key, but
    // not the dipole orientation (the width's error does not depend on it, and a batch of dipoles
    // has one axis per member); the class is tuned with its first member's axis
    std::vector<std::string> keys;
    std::vector<nlint_params> ctuned;
    std::vector<nlint_tune_report> creps;
    std::vector<int> cls((size_t)count);
    for (int i = 0; i < count; i++) {
        nlint_params p = in[i];
        if (p.precision != NLINT_FP32 && p.precision != NLINT_FP64)
            p.precision = tol >= 1e-7 ? NLINT_FP32 : NLINT_FP64;
        for (int k = 0; k < 3; k++) p.axis[k] = p.axis2[k] = 0.0;
        const std::string key = cache_key(p, tol);
        size_t c = 0;
        while (c < keys.size() && keys[c] != key) c++;
        if (c == keys.size()) {
            nlint_params t;
            nlint_tune_report r;
            const int rc = nlint_autotune(&in[i], tol, cache_path, &t, &r);
            if (rc) return rc;
            keys.push_back(key);
            ctuned.push_back(t);
            creps.push_back(r);
        }
        cls[(size_t)i] = (int)c;
    }
    // the three parameter sets; each member keeps its own axis and density
    std::vector<nlint_params> cand[3];
    bool any_alt = false;
    for (int i = 0; i < count; i++) {
        const nlint_params &t = ctuned[(size_t)cls[(size_t)i]];
        nlint_params p = in[i];
        p.precision = t.precision;
        p.w = t.w;
        p.bin_shape = t.bin_shape;
        p.max_sub = t.max_sub;
        p.fft_sched = t.fft_sched;  // the class's FFT schedules in every set
        cand[0].push_back(p);
        p.bin_shape = 0;
        p.max_sub = 0;
        cand[1].push_back(p);
        const int wa = creps[(size_t)cls[(size_t)i]].w_alt;
        if (wa > 0) {
            p.w = wa;
            any_alt = true;
        }
        cand[2].push_back(p);
    }
    if (in[0].device >= 0 && cudaSetDevice(in[0].device) != cudaSuccess)
        return tfail(NLINT_ECUDA, "autotune_batch: cudaSetDevice failed");
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        return tfail(NLINT_ECUDA, "autotune_batch: stream creation failed");
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{s};
    double ms[3] = {0.0, 0.0, 0.0};
    int choice = 0;
    for (int k = 0; k < (any_alt ? 3 : 2); k++) {
        const int rc = time_batch(cand[k], branches, 5, s, ms[k]);
        if (rc) return rc;
        if (ms[k] < ms[choice]) choice = k;
    }
    for (int i = 0; i < count; i++) {
        out[i] = cand[choice][(size_t)i];
        if (member_reps) {
            nlint_tune_report r = creps[(size_t)cls[(size_t)i]];
            if (out[i].w != r.w) {  // the alternative width was kept: report it as the choice
                std::swap(r.w, r.w_alt);
                std::swap(r.err, r.err_alt);
            }
            r.bin_shape = out[i].bin_shape;
            r.max_sub = out[i].max_sub;
            member_reps[i] = r;
        }
    }
    if (rep) *rep = nlint_batch_tune_report{choice, (int)keys.size(), {ms[0], ms[1], ms[2]}};
    return NLINT_OK;
}
