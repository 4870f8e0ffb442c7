// Plan builder and C-ABI entry points.
//
// The plan follows Algorithm 1 (Section 3.2): steps 1-3 (grid, nodes and weights of
// eq. 3.7) run once on the host in FP64; steps 4-5 (type-2 NUFFT, multiply, type-1 NUFFT)
// and the energy of Remark 3.3 run on the device for every evaluation.  Besides that path:
// Algorithm 2 (Section 3.3, run_alg2), the same operator with its Toeplitz kernel precomputed
// (nlint_plan_toeplitz), the stage entry points, and the host-buffer forms (nlint_eval_host,
// and nlint_eval_host_many with its copies overlapped with the evaluations).  An Algorithm 1
// plan clears its spread grid on a side stream while the interpolation runs.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace nlint {

static thread_local std::string g_err;

static void fit_phi_poly(nlint_plan_s *p);
static int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}
// Records a failure message for nlint_last_error from other translation units.
int report_error(int code, const char *msg) { return fail(code, msg); }

static int cuda_fail(cudaError_t e, const char *where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return NLINT_ECUDA;
}
#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

// ------------------------------------------------------------------ Gauss-Legendre (FP64)
// m-point rule on [-1, 1]: Newton's method on P_m, with P_m and P_m' from the three-term
// recurrence (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}.
static void gauss_legendre(int m, std::vector<double> &x, std::vector<double> &w) {
    x.assign(m, 0.0);
    w.assign(m, 0.0);
    for (int i = 0; i < (m + 1) / 2; i++) {
        double z = std::cos(M_PI * (i + 0.75) / (m + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int j = 1; j < m; j++) {
                double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            if (m == 1) { p1 = z; p0 = 1.0; }
            dp = m * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int j = 1; j < m; j++) {
            double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
            p0 = p1;
            p1 = p2;
        }
        // (1 - z)(1 + z) in place of 1 - z^2: no cancellation next to the ends of [-1, 1]
        dp = m * (p0 - z * p1) / ((1.0 - z) * (1.0 + z));
        x[i] = -z;
        x[m - 1 - i] = z;
        w[i] = w[m - 1 - i] = 2.0 / ((1.0 - z) * (1.0 + z) * dp * dp);
    }
}


std::vector<int16_t> build_pair_order(int w, int row, int banks, int lanes, int group) {
    std::vector<std::pair<int, int>> rest;
    for (int a = 0; a < w; a++)
        for (int b = 0; b < w; b++) rest.push_back({a, b});
    const int passes = (w * w + lanes - 1) / lanes;
    if (group <= 0 || group > lanes) group = lanes;
    std::vector<int16_t> out((size_t)passes * lanes, (int16_t)-1);
    for (int ps = 0; ps < passes; ps++) {
        // lanes in groups served by one shared-memory wavefront: distinct banks within a group
        for (int g0 = 0; g0 < lanes && !rest.empty(); g0 += group) {
            std::vector<std::pair<int, int>> cur, later;
            std::vector<bool> used(banks, false);
            for (auto &q : rest) {
                const int r = (q.first * row + q.second) % banks;
                if ((int)cur.size() < group && !used[r]) {
                    used[r] = true;
                    cur.push_back(q);
                } else {
                    later.push_back(q);
                }
            }
            while ((int)cur.size() < group && !later.empty()) {  // a bank is shared: unavoidable
                cur.push_back(later.front());
                later.erase(later.begin());
            }
            for (size_t l = 0; l < cur.size(); l++)
                out[(size_t)ps * lanes + g0 + l] = (int16_t)(cur[l].first << 8 | cur[l].second);
            rest = later;
        }
    }
    return out;
}

void build_node_groups(const int32_t *org, int64_t first, int64_t count, int lanes, int banks,
                       std::vector<int64_t> &order, std::vector<int> &sizes) {
    struct Run {
        int32_t o;
        int64_t next, end;
    };
    std::vector<Run> runs;  // runs of one origin (the nodes are sorted by origin)
    for (int64_t i = first; i < first + count;) {
        int64_t k = i;
        while (k < first + count && org[k] == org[i]) k++;
        runs.push_back({org[i], i, k});
        i = k;
    }
    std::stable_sort(runs.begin(), runs.end(),
                     [](const Run &a, const Run &b) { return a.end - a.next > b.end - b.next; });
    size_t head = 0;  // runs before head are used up
    int64_t left = count;
    while (left > 0) {
        int32_t owner[32];
        for (int r = 0; r < 32; r++) owner[r] = -1;  // origin offsets are >= 0
        int slots = lanes;
        while (head < runs.size() && runs[head].next == runs[head].end) head++;
        for (size_t u = head; u < runs.size() && slots > 0; u++) {
            Run &ru = runs[u];
            if (ru.next == ru.end) continue;
            const int r = ru.o % banks;
            if (owner[r] >= 0 && owner[r] != ru.o) continue;
            owner[r] = ru.o;
            const int64_t take = std::min<int64_t>(slots, ru.end - ru.next);
            for (int64_t t = 0; t < take; t++) order.push_back(ru.next + t);
            ru.next += take;
            slots -= (int)take;
        }
        sizes.push_back(lanes - slots);
        left -= lanes - slots;
    }
}

// A tiled tensor map of the stored half of the fine grid G (n x n x (n/2 + 1) complex floats,
// handled as 8-byte cells, x fastest) with boxes of T[2] x T[1] x T[0] cells, for TMA loads of
// the interpolation's tiles.  cuTensorMapEncodeTiled is reached through the runtime's driver
// entry points (the library does not link the driver library).  false: no tensor map (the
// kernels then stage by plain loads).
typedef CUresult (*tmap_encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);

bool encode_grid_tmap(CUtensorMap *map, void *G, int n, const int *T) {
    static tmap_encode_fn encode = nullptr;
    if (!encode) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !f) {
            (void)cudaGetLastError();
            return false;
        }
        encode = (tmap_encode_fn)f;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)(n / 2 + 1)};
    const cuuint64_t strides[2] = {(cuuint64_t)n * 8, (cuuint64_t)n * n * 8};  // bytes, dims 1 and 2
    const cuuint32_t box[3] = {(cuuint32_t)T[2], (cuuint32_t)T[1], (cuuint32_t)T[0]};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (box[0] > 256 || box[1] > 256 || box[2] > 256 || (box[0] * 8) % 16 != 0) return false;
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, G, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace nlint

// ---------------------------------------------------------------------------------- plan
struct nlint_plan_s {
    nlint_params prm;
    int d, prec, w, pad, n_fine;
    int64_t N, nr, nt, nphi, Nf, Mh;
    double L, h, P, sigma, beta;
    double axis[3], axis2[3], alpha;
    int device;
    // device memory
    int32_t *d_rel = nullptr;
    int4 *d_pos = nullptr;       // FP32 plans: per-node origin and offset records
    void *d_ker = nullptr, *d_W = nullptr, *d_fac = nullptr, *d_tw = nullptr;
    int32_t *d_perm = nullptr, *d_mirror = nullptr;
    int4 *d_subs = nullptr, *d_bins = nullptr;
    int4 *d_gsubs = nullptr;     // FP32 3D: interpolation subproblems over node groups
    CUtensorMap tmapG;           // FP32 3D Algorithm 1: the fine grid as a TMA tensor (has_tmap)
    bool has_tmap = false;
    int *d_status = nullptr;     // bit 0: a bounded device-side wait ran out
    int32_t *d_grp = nullptr;    // FP32 3D: first node of each group (and one past the last)
    int16_t *d_pairs = nullptr, *d_pairs_i = nullptr;  // spreading / interpolation lane tables
    double2 *d_epart = nullptr;  // energy-only path: one partial per subproblem
    int32_t *d_crowd_bin = nullptr;
    double2 *d_crowd = nullptr;
    int B[3], T[3];
    int bin_shape = 1;
    unsigned fft_sched = 0;      // FFT pass schedules (nlint_params.fft_sched; FP32 only)
    int phpoly = 0;              // FP32 3D, w >= 7: stencil-value polynomials (fit_phi_poly)
    float phc[nlint::NODE_MAXW * nlint::PH_NC] = {};
    int64_t nsub = 0, nbins = 0, ngsub = 0;
    int ncrowd = 0;
    size_t bytes_crowd = 0;
    void *d_bufA = nullptr, *d_bufB = nullptr, *d_bufG = nullptr, *d_c = nullptr;
    // Algorithm 1: the spread grid in its own buffer, cleared on a side stream while the
    // interpolation runs (NULL: the spreading clears d_bufG in stream order)
    void *d_bufH = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_zero = nullptr;
    double2 *d_partials = nullptr;
    double *d_E = nullptr;
    void *d_rho_io = nullptr, *d_u_io = nullptr;  // nlint_eval_host staging
    // nlint_eval_host_many: two staging buffers each way, a copy-in and a copy-out stream, the
    // events that order them against the evaluations, and the energies on the device
    void *d_rho_st[2] = {nullptr, nullptr}, *d_u_st[2] = {nullptr, nullptr};
    double *d_Em = nullptr;
    int64_t nEm = 0;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_io[7] = {};  // in[2], comp[2], out[2], fork/join
    int n_partials = 0;
    size_t bytes_A = 0, bytes_B = 0, bytes_G = 0, bytes_Hext = 0, bytes_c = 0;
    size_t ws_bytes = 0;
    nlint::PassDesc P1, P2, P3, Q1, Q2, Q3;
    // precomputed Toeplitz kernel (nlint_plan_toeplitz): K_hat on the Hermitian half grid
    void *d_fac1 = nullptr, *d_khat = nullptr;
    bool toeplitz = false;
    nlint::PassDesc T1, U3;
    nlint::PassDesc X;  // forward FFT along x, multiply by K_hat, inverse FFT (one row pass)
    // Algorithm 2 (eq. 3.9): I_1's multiplier U_hat (1 - p) lives in d_khat and uses the
    // T1/X/U3 passes; the node set is I_2's (radius P2, weights times p)
    int algorithm = 1;
    double pu_a = 0.0, pu_r0 = 0.0, pu_r1 = 0.0, rad2 = 0.0;  // rad2: I_2's radius P2
    // I_2's frequency window: its nodes' stencils lie within |l_a| <= win fine cells, so its
    // FFT passes transform only the window's lines (0 = the full passes P1..Q3)
    int win = 0;
    int64_t ball2 = 0;      // ball window of the full x passes (PassDesc::ball2)
    int64_t conv_ball2 = 0; // Algorithm 2: rows of I_1's convolution pass beyond it are zero
    size_t bytes_Hwin = 0;  // the planes of the spread grid the window touches
    nlint::PassDesc P1w, P2w, P3w, Q1w, Q2w, Q3w;
    // dual z passes shared by I_1 and I_2 (the first forward one reads the density once for both,
    // the last inverse one writes u once); d_win holds I_2's window planes meanwhile
    bool dual = false;
    nlint::PassDesc D6, D7;
    void *d_win = nullptr;
    size_t bytes_win = 0;
    // host copies for inspection (canonical order)
    std::vector<double> k_canon, W_canon;
    // stage timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    std::vector<const char *> ev_names;
    int ev_used = 0;
    int64_t launches = 0;  // kernels this plan has launched (all entry points)
};

namespace nlint {

static int64_t default_nr(int d, int64_t n) {
    if (d == 2) return std::max<int64_t>(8, n / 4);
    double v;
    if (n <= 32) v = (double)n;
    else if (n <= 128) v = 32.0 + (n - 32) * (64.0 / 96.0);
    else if (n <= 256) v = 96.0 + (n - 128) * (64.0 / 128.0);
    else v = 160.0 + (n - 256) * 0.5;
    int64_t r = (int64_t)std::llround(v / 8.0) * 8;
    return std::max<int64_t>(8, r);
}

// Kernel symbols of table int3dd: eqs. Cou3D, Cou2D, dipkerneldF (dipkernelF when m = n) and
// dipkernelF2dd (dipkernelF2d when m = n); n = axis, m = axis2, both unit vectors.
static double u_hat(const nlint_plan_s *p, const double k[3]) {
    const double k2 = k[0] * k[0] + k[1] * k[1] + (p->d == 3 ? k[2] * k[2] : 0.0);
    if (p->prm.kernel == NLINT_COULOMB) return p->d == 3 ? 1.0 / k2 : 1.0 / std::sqrt(k2);
    const double *n = p->axis, *m = p->axis2;
    if (p->d == 3) {
        const double kn = k[0] * n[0] + k[1] * n[1] + k[2] * n[2];
        const double km = k[0] * m[0] + k[1] * m[1] + k[2] * m[2];
        const double mn = m[0] * n[0] + m[1] * n[1] + m[2] * n[2];
        return -mn + 3.0 * kn * km / k2;
    }
    const double kn = k[0] * n[0] + k[1] * n[1], km = k[0] * m[0] + k[1] * m[1];
    return -p->alpha + 3.0 * (kn * km - n[2] * m[2] * k2) / (2.0 * std::sqrt(k2));
}

// Partition of unity of Algorithm 2: p_3(k) = exp(-|k|^2 / a) (eq. 3.10),
// p_2(k) = erfc(12 (|k| - (R0 + R1)/2) / (R1 - R0)) / 2 (eq. 3.12).
static double partition(const nlint_plan_s *p, const double k[3]) {
    const double k2 = k[0] * k[0] + k[1] * k[1] + (p->d == 3 ? k[2] * k[2] : 0.0);
    if (p->d == 3) return std::exp(-k2 / p->pu_a);
    return 0.5 * std::erfc(12.0 * (std::sqrt(k2) - 0.5 * (p->pu_r0 + p->pu_r1)) / (p->pu_r1 - p->pu_r0));
}

// I_1's multiplier of Algorithm 2 (eq. 3.9, step 3): M(k) = U_hat(k) (1 - p(k)) on the closed
// ball |k| <= P (a relative margin of 1e-12 keeps the sphere's lattice points), 0 outside.  At
// k = 0 the symbol takes its limit: 1/a for the 3D Coulomb kernel ((1 - e^{-k^2/a}) / k^2),
// 0 otherwise (1 - p_3 ~ k^2/a against a bounded dipole symbol; 1 - p_2(0) is below rounding).
static double alg2_multiplier(const nlint_plan_s *p, const double k[3]) {
    const double k2 = k[0] * k[0] + k[1] * k[1] + (p->d == 3 ? k[2] * k[2] : 0.0);
    const double pm = p->P * (1.0 + 1e-12);
    if (k2 > pm * pm) return 0.0;
    if (k2 == 0.0) return (p->d == 3 && p->prm.kernel == NLINT_COULOMB) ? 1.0 / p->pu_a : 0.0;
    const double one_minus_p = p->d == 3 ? -std::expm1(-k2 / p->pu_a) : 1.0 - partition(p, k);
    return u_hat(p, k) * one_minus_p;
}

// Fourier transform of the ES kernel, Phi(xi) = int_{-1}^{1} phi(z) cos(xi z) dz, by a
// 256-point Gauss-Legendre rule in FP64.
static double es_ft(double xi, double beta, const std::vector<double> &qx,
                    const std::vector<double> &qw) {
    double s = 0.0;
    for (size_t i = 0; i < qx.size(); i++) {
        const double z = qx[i];
        const double ph = std::exp(beta * (std::sqrt(std::max(0.0, 1.0 - z * z)) - 1.0));
        s += qw[i] * ph * std::cos(xi * z);
    }
    return s;
}

template <typename T>
static std::vector<T> cast_vec(const std::vector<double> &v) {
    std::vector<T> o(v.size());
    for (size_t i = 0; i < v.size(); i++) o[i] = (T)v[i];
    return o;
}

template <typename T>
static int upload(void **dst, const std::vector<double> &v, size_t &acc) {
    std::vector<T> h = cast_vec<T>(v);
    size_t b = h.size() * sizeof(T);
    if (b == 0) b = sizeof(T);
    CK(cudaMalloc(dst, b));
    acc += b;
    if (!h.empty()) CK(cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return NLINT_OK;
}

static void plan_free(nlint_plan_s *p) {
    void *ptrs[] = {p->d_rel, p->d_pos, p->d_gsubs, p->d_grp, p->d_status, p->d_ker, p->d_W, p->d_fac, p->d_tw, p->d_perm, p->d_mirror,
                    p->d_subs, p->d_bins, p->d_crowd_bin, p->d_crowd, p->d_pairs, p->d_pairs_i, p->d_epart, p->d_fac1, p->d_khat,
                    p->d_win, p->d_bufA, p->d_bufB, p->d_bufG, p->d_bufH, p->d_c, p->d_partials, p->d_E,
                    p->d_rho_io, p->d_u_io, p->d_rho_st[0], p->d_rho_st[1], p->d_u_st[0],
                    p->d_u_st[1], p->d_Em};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_zero) cudaEventDestroy(p->ev_zero);
    if (p->side) cudaStreamDestroy(p->side);
    for (cudaEvent_t e : p->ev_io)
        if (e) cudaEventDestroy(e);
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_out) cudaStreamDestroy(p->s_out);
}

static int alg2_setup(nlint_plan_s *p);

static int build_plan(const nlint_params *in, nlint_plan_s *p) {
    p->prm = *in;
    const nlint_params &q = *in;
    if (q.d != 2 && q.d != 3) return fail(NLINT_EINVAL, "d must be 2 or 3");
    if (q.n < 8 || q.n % 2) return fail(NLINT_EINVAL, "n must be even and >= 8");
    if (!(q.L > 0.0) || !std::isfinite(q.L)) return fail(NLINT_EINVAL, "L must be positive");
    if (q.kernel != NLINT_COULOMB && q.kernel != NLINT_DIPOLE)
        return fail(NLINT_EINVAL, "kernel must be NLINT_COULOMB or NLINT_DIPOLE");
    if (q.max_sub < 0 || q.max_sub > (1 << 20)) return fail(NLINT_EINVAL, "max_sub must be in [0, 2^20]");
    if (q.crowd_min < 0) return fail(NLINT_EINVAL, "crowd_min must be >= 0");
    if (q.fft_sched < 0 || q.fft_sched > 15) return fail(NLINT_EINVAL, "fft_sched must be in [0, 15]");
    p->d = q.d;
    p->N = q.n;
    p->L = q.L;
    p->h = q.L / (double)q.n;
    p->alpha = 0.0;
    if (q.kernel == NLINT_DIPOLE) {
        const double nn = std::sqrt(q.axis[0] * q.axis[0] + q.axis[1] * q.axis[1] + q.axis[2] * q.axis[2]);
        if (!(nn > 0.0) || !std::isfinite(nn)) return fail(NLINT_EINVAL, "dipole axis must be non-zero");
        for (int a = 0; a < 3; a++) p->axis[a] = q.axis[a] / nn;
        const double mm = std::sqrt(q.axis2[0] * q.axis2[0] + q.axis2[1] * q.axis2[1] + q.axis2[2] * q.axis2[2]);
        if (!std::isfinite(mm)) return fail(NLINT_EINVAL, "second dipole axis must be finite");
        for (int a = 0; a < 3; a++) p->axis2[a] = mm > 0.0 ? q.axis2[a] / mm : p->axis[a];
        if (!std::isfinite(q.alpha)) return fail(NLINT_EINVAL, "alpha must be finite");
        if (q.d == 2) p->alpha = q.alpha;
    } else {
        for (int a = 0; a < 3; a++) p->axis[a] = p->axis2[a] = 0.0;
    }
    const double pmax = M_PI / p->h;
    p->P = (q.P > 0.0) ? q.P : pmax;
    if (p->P > pmax * (1.0 + 1e-12))
        return fail(NLINT_EINVAL, "P must not exceed pi/h (nodes beyond the grid's Nyquist radius)");
    p->algorithm = q.algorithm == 0 ? 1 : q.algorithm;
    if (p->algorithm != 1 && p->algorithm != 2) return fail(NLINT_EINVAL, "algorithm must be 1 or 2");
    if (p->algorithm == 2) {
        // partition of unity (eq. 3.9): p_3 = exp(-|k|^2/a) (eq. 3.10), p_2 of eq. 3.12
        if (!(q.pu_a >= 0.0) || !(q.pu_r0 >= 0.0) || !(q.pu_r1 >= 0.0) || !(q.P2 >= 0.0) ||
            !std::isfinite(q.pu_a) || !std::isfinite(q.pu_r0) || !std::isfinite(q.pu_r1) || !std::isfinite(q.P2))
            return fail(NLINT_EINVAL, "Algorithm 2 parameters (pu_a, pu_r0, pu_r1, P2) must be finite and >= 0");
        if (q.d == 3) {
            p->pu_a = q.pu_a > 0.0 ? q.pu_a : (11.8 / q.L) * (11.8 / q.L);
            p->rad2 = std::min(p->P, 6.1 * std::sqrt(p->pu_a));
        } else {
            p->pu_r0 = q.pu_r0 > 0.0 ? q.pu_r0 : 12.0 / q.L;
            p->pu_r1 = q.pu_r1 > 0.0 ? q.pu_r1 : 160.0 / q.L;
            if (!(p->pu_r1 > p->pu_r0)) return fail(NLINT_EINVAL, "Algorithm 2 needs pu_r0 < pu_r1");
            p->rad2 = std::min(p->P, p->pu_r1);
        }
        if (q.P2 > 0.0) p->rad2 = q.P2;
        if (p->rad2 > p->P * (1.0 + 1e-12)) return fail(NLINT_EINVAL, "P2 must not exceed P");
    }
    double eps = q.eps > 0.0 ? q.eps : 1e-6;
    if (eps < 1e-15) eps = 1e-15;
    p->prec = (q.precision == NLINT_FP32 || q.precision == NLINT_FP64) ? q.precision
                                                                       : (eps >= 1e-7 ? NLINT_FP32 : NLINT_FP64);
    p->fft_sched = p->prec == NLINT_FP32 ? (unsigned)q.fft_sched : 0u;
    int w = q.w > 0 ? q.w : (int)std::ceil(-std::log10(eps)) + 1;
    if (w < 2) w = 2;
    if (w > 16) return fail(NLINT_EINVAL, "spreading width must be <= 16");
    p->w = w;
    p->sigma = q.sigma > 0.0 ? q.sigma : 2.0;
    if (p->sigma < 1.25) return fail(NLINT_EINVAL, "sigma must be >= 1.25");
    const int64_t nf = fft_next_size((int64_t)std::ceil(p->sigma * (double)p->N));
    if (nf < 0) return fail(NLINT_EUNSUPPORTED, "fine grid larger than 2048 per axis");
    p->n_fine = (int)nf;
    p->pad = w / 2 + 1;
    if (p->n_fine < 4 * p->pad + 2)
        return fail(NLINT_EUNSUPPORTED, "grid too small for this spreading width (n_fine < 4*(w/2+1)+2)");
    const double sig_eff = (double)p->n_fine / (double)p->N;
    p->beta = 0.97 * M_PI * (1.0 - 1.0 / (2.0 * sig_eff)) * w;  // ES shape parameter
    fit_phi_poly(p);

    const int64_t nr_alg2 = p->d == 3 ? (p->prec == NLINT_FP32 ? 32 : 40) : (p->prec == NLINT_FP32 ? 48 : 64);
    p->nr = q.n_r > 0 ? q.n_r : (p->algorithm == 2 ? nr_alg2 : default_nr(p->d, p->N));
    if (p->d == 3) {
        p->nt = q.n_theta > 0 ? q.n_theta : p->nr;
        p->nphi = q.n_phi > 0 ? q.n_phi : 2 * p->nr;
    } else {
        p->nt = 1;
        p->nphi = q.n_phi > 0 ? q.n_phi : 2 * p->nr;
    }
    if (p->nphi % 2) return fail(NLINT_EINVAL, "n_phi must be even (the node set must be symmetric)");
    if (p->d == 3 && p->nt % 2) return fail(NLINT_EINVAL, "n_theta must be even");
    p->Nf = p->nr * p->nt * p->nphi;
    p->Mh = p->Nf / 2;
    if (p->Nf > (int64_t)2000000000) return fail(NLINT_EUNSUPPORTED, "too many nodes");

    int dev = q.device;
    if (dev < 0) CK(cudaGetDevice(&dev));
    CK(cudaSetDevice(dev));
    p->device = dev;

    // ---------------- nodes and weights (eq. 3.7), FP64, canonical order
    std::vector<double> xr, wr, xt, wt;
    gauss_legendre((int)p->nr, xr, wr);
    const double Prad = p->algorithm == 2 ? p->rad2 : p->P;  // Algorithm 2: I_2's nodes
    for (auto &v : xr) v = Prad * (1.0 + v) / 2.0;
    for (auto &v : wr) v = Prad * v / 2.0;
    if (p->d == 3) {
        gauss_legendre((int)p->nt, xt, wt);
        for (auto &v : xt) v = M_PI * (1.0 + v) / 2.0;
        for (auto &v : wt) v = M_PI * v / 2.0;
    }
    const double wphi = 2.0 * M_PI / (double)p->nphi;
    const double twopi_d = std::pow(2.0 * M_PI, p->d);
    p->k_canon.assign((size_t)p->Nf * p->d, 0.0);
    p->W_canon.assign((size_t)p->Nf, 0.0);
    for (int64_t a = 0; a < p->nr; a++)
        for (int64_t b = 0; b < p->nt; b++)
            for (int64_t c = 0; c < p->nphi; c++) {
                const int64_t j = (a * p->nt + b) * p->nphi + c;
                const double r = xr[a], ph = wphi * (double)c;
                double k[3] = {0, 0, 0}, wj;
                if (p->d == 3) {
                    const double st = std::sin(xt[b]), ct = std::cos(xt[b]);
                    k[0] = r * st * std::cos(ph);
                    k[1] = r * st * std::sin(ph);
                    k[2] = r * ct;
                    wj = wr[a] * wt[b] * st * wphi * r * r;
                } else {
                    k[0] = r * std::cos(ph);
                    k[1] = r * std::sin(ph);
                    wj = wr[a] * wphi * r;
                }
                for (int e = 0; e < p->d; e++) p->k_canon[(size_t)j * p->d + e] = k[e];
                p->W_canon[j] = wj * u_hat(p, k) / twopi_d;
                if (p->algorithm == 2) p->W_canon[j] *= partition(p, k);
            }

    // ---------------- half node set, stencil origins, tile sort
    const int64_t Mh = p->Mh;
    std::vector<int64_t> half(Mh), mir(Mh);
    {
        int64_t o = 0;
        for (int64_t a = 0; a < p->nr; a++)
            for (int64_t b = 0; b < p->nt; b++)
                for (int64_t c = 0; c < p->nphi; c++) {
                    const bool keep = (p->d == 3) ? (b < p->nt / 2) : (c < p->nphi / 2);
                    if (!keep) continue;
                    const int64_t j = (a * p->nt + b) * p->nphi + c;
                    const int64_t bm = (p->d == 3) ? (p->nt - 1 - b) : 0;
                    const int64_t cm = (c + p->nphi / 2) % p->nphi;
                    half[o] = j;
                    mir[o] = (a * p->nt + bm) * p->nphi + cm;
                    o++;
                }
    }
    const int d = p->d, n = p->n_fine;
    const double gscale = p->h * (double)n / (2.0 * M_PI);
    std::vector<int32_t> l0((size_t)d * Mh);
    std::vector<double> fr((size_t)d * Mh);
    int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    int64_t ball2 = 0;  // max over the nodes of the squared norm of their farthest stencil cell
    for (int64_t o = 0; o < Mh; o++) {
        const int64_t j = half[o];
        int64_t r2 = 0;
        for (int ax = 0; ax < d; ax++) {
            // array axis ax pairs with node component d-1-ax (axis 0 is k_z in 3D, k_y in 2D)
            const double g = p->k_canon[(size_t)j * d + (d - 1 - ax)] * gscale;
            const int32_t l = (int32_t)std::ceil(g - 0.5 * w);
            l0[(size_t)ax * Mh + o] = l;
            fr[(size_t)ax * Mh + o] = g - (double)l;
            if (ax == 0 && (l < -p->pad || l + w - 1 > n / 2 + p->pad))
                return fail(NLINT_EINVAL, "internal: node stencil outside the stored half grid");
            lo[ax] = std::min(lo[ax], l);
            hi[ax] = std::max(hi[ax], l);
            const int64_t far = std::max(std::abs((int64_t)l), std::abs((int64_t)l + w - 1));
            r2 += far * far;
        }
        ball2 = std::max(ball2, r2);
    }
    // (a signed FFT index never exceeds the unwrapped cell index in magnitude, so the bound
    // holds for the stored grid too); a ball that covers the whole grid is no window
    p->ball2 = (ball2 < (int64_t)d * (n / 2) * (n / 2)) ? ball2 : 0;
    // 3D: bins start at even cells along axis 2 (the spreading's tile flush adds two adjacent
    // cells per 16-byte vector atomic, which must start at an even grid index)
    if (d == 3 && Mh) lo[2] -= lo[2] & 1;
    // bins: boxes of B[ax] stencil-origin cells starting at lo[ax]; tile = B + w - 1.  The
    // shape is a plan parameter (the autotuner searches it); an automatic choice whose tile
    // does not fit in shared memory at this width falls back to the smallest shape
    {
        const bool f64 = p->prec == NLINT_FP64;
        int bs = q.bin_shape > 0 ? q.bin_shape : default_bin_shape(f64, d, w);
        if (!bin_shape_built(f64, d, bs))
            return fail(NLINT_EINVAL, "bin shape not available for this precision and dimension "
                                      "(3D FP32: 1, 3, 4; 3D FP64: 1, 2; 2D: 1)");
        if (node_smem_for(p->prec, d, w, bs) > NODE_SMEM_MAX) {
            if (q.bin_shape > 0)
                return fail(NLINT_EUNSUPPORTED, "the bin shape's tile does not fit in shared memory at this width");
            bs = (d == 3 && f64) ? 2 : 1;
        }
        p->bin_shape = bs;
    }
    for (int ax = 0; ax < 3; ax++) {
        p->B[ax] = 1;
        p->T[ax] = 1;
    }
    for (int ax = 0; ax < d; ax++) {
        const int b = bin_dim(d, p->bin_shape, ax);
        p->B[ax] = b;
        p->T[ax] = b + w - 1;
    }
    int64_t nbin[3] = {1, 1, 1};
    for (int ax = 0; ax < d; ax++) nbin[ax] = (Mh ? (hi[ax] - lo[ax]) / p->B[ax] + 1 : 1);
    // sort by bin, then by stencil origin inside the bin (a warp's consecutive nodes then touch
    // overlapping tile cells), then canonical order
    std::vector<int64_t> key(Mh), okey(Mh);
    for (int64_t o = 0; o < Mh; o++) {
        int64_t kk = 0, oo = 0;
        for (int ax = 0; ax < d; ax++) {
            const int32_t rel = l0[(size_t)ax * Mh + o] - lo[ax];
            kk = kk * nbin[ax] + rel / p->B[ax];
            oo = oo * p->B[ax] + rel % p->B[ax];
        }
        key[o] = kk;
        okey[o] = oo;
    }
    std::vector<int64_t> ord(Mh);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
        return key[a] != key[b] ? key[a] < key[b] : okey[a] < okey[b];
    });
    // FP32 3D: each bin's nodes in lane groups for the interpolation (build_node_groups); the
    // groups keep nodes of one origin together, so the spreading still meets them in pairs
    const bool grouped = p->prec == NLINT_FP32 && d == 3;
    std::vector<int> gsize;          // node count of each group, bins in order
    std::vector<int64_t> gbin_end;   // one past each bin's last group
    if (grouped) {
        // the interpolation's tile: 8-byte complex cells, rows of T2 cells (no padding: the
        // lanes of a warp read one offset from their own origins, so only the origins matter)
        const int T1 = p->B[1] + w - 1;
        const int P2 = p->B[2] + w - 1;
        std::vector<int32_t> org(Mh);
        for (int64_t o = 0; o < Mh; o++) {
            const int64_t sidx = ord[o];
            int32_t r[3];
            for (int ax = 0; ax < 3; ax++) r[ax] = (l0[(size_t)ax * Mh + sidx] - lo[ax]) % p->B[ax];
            org[o] = (r[0] * T1 + r[1]) * P2 + r[2];
        }
        std::vector<int64_t> neworder;
        neworder.reserve(Mh);
        for (int64_t o = 0; o < Mh;) {
            int64_t e = o;
            while (e < Mh && key[ord[e]] == key[ord[o]]) e++;
            build_node_groups(org.data(), o, e - o, 16, 16, neworder, gsize);
            if (gsize.size() & 1) gsize.push_back(0);  // half-groups pair up within a bin
            gbin_end.push_back((int64_t)gsize.size());
            o = e;
        }
        std::vector<int64_t> ord2(Mh);
        for (int64_t o = 0; o < Mh; o++) ord2[o] = ord[neworder[o]];
        ord.swap(ord2);
    }
    std::vector<int32_t> l0s((size_t)d * Mh), perm(Mh), mirror(Mh);
    std::vector<double> frs((size_t)d * Mh), Ws(Mh);
    const double hd = std::pow(p->h, d);
    for (int64_t o = 0; o < Mh; o++) {
        const int64_t s = ord[o];
        for (int ax = 0; ax < d; ax++) {
            l0s[(size_t)ax * Mh + o] = l0[(size_t)ax * Mh + s];
            frs[(size_t)ax * Mh + o] = fr[(size_t)ax * Mh + s];
        }
        perm[o] = (int32_t)half[s];
        mirror[o] = (int32_t)mir[s];
        Ws[o] = hd * p->W_canon[half[s]];
    }
    // non-empty bins and their subproblems; crowded bins (FP32 plans) are summed in FP64
    const int max_sub = q.max_sub > 0 ? q.max_sub : ((p->prec == NLINT_FP32) ? 1024 : 512);
    const int max_sub_crowd = std::min(max_sub, 512);
    const int64_t crowd_min = q.crowd_min > 0 ? q.crowd_min : 4096;
    std::vector<int4> bins, subs;
    std::vector<int32_t> rel(Mh);
    std::vector<int32_t> crowd_bin;
    for (int64_t o = 0; o < Mh;) {
        int64_t e = o;
        while (e < Mh && key[ord[e]] == key[ord[o]]) e++;
        int4 b;
        const int64_t kk = key[ord[o]];
        int64_t rem = kk;
        int org[3] = {0, 0, 0};
        for (int ax = d - 1; ax >= 0; ax--) {
            org[ax] = lo[ax] + (int)(rem % nbin[ax]) * p->B[ax];
            rem /= nbin[ax];
        }
        b.x = org[0];
        b.y = org[1];
        b.z = org[2];
        for (int64_t q = o; q < e; q++) {  // stencil origins relative to the bin
            int32_t r = 0;
            for (int ax = 0; ax < d; ax++) r |= (l0s[(size_t)ax * Mh + q] - org[ax]) << (8 * ax);
            rel[q] = r;
        }
        const bool crowd = (p->prec == NLINT_FP32) && (e - o > crowd_min);
        b.w = crowd ? (int)crowd_bin.size() : -1;
        const int bi = (int)bins.size();
        if (crowd) crowd_bin.push_back(bi);
        bins.push_back(b);
        const int cap = crowd ? max_sub_crowd : max_sub;
        const int64_t nsub = (e - o + cap - 1) / cap;
        for (int64_t q = 0; q < nsub; q++) {
            const int64_t a = o + (e - o) * q / nsub, z = o + (e - o) * (q + 1) / nsub;
            subs.push_back(make_int4((int)a, (int)(z - a), bi, 0));
        }
        o = e;
    }
    p->nsub = (int64_t)subs.size();
    p->nbins = (int64_t)bins.size();
    p->ncrowd = (int)crowd_bin.size();
    if (p->nsub > (int64_t)INT32_MAX) return fail(NLINT_EUNSUPPORTED, "too many subproblems");
    // the interpolation's subproblems: runs of at most max_sub / 16 half-group pairs of one bin
    // (up to 2 max_sub nodes: a crowded bin's tile is staged half as often as the spreading's;
    // 256^3 FP32: 2.17 -> 2.14 ms per evaluation against max_sub / 32)
    std::vector<int32_t> grp;
    std::vector<int4> gsubs;
    if (grouped) {
        grp.resize(gsize.size() + 1);
        grp[0] = 0;
        for (size_t g = 0; g < gsize.size(); g++) grp[g + 1] = grp[g] + gsize[g];
        const int64_t gmax = std::max(1, max_sub / 16);
        int64_t g0 = 0;
        for (size_t bi = 0; bi < bins.size(); bi++) {  // in pairs of half-groups
            const int64_t g1 = gbin_end[bi] / 2, ng = g1 - g0, ns = (ng + gmax - 1) / gmax;
            for (int64_t qq = 0; qq < ns; qq++) {
                const int64_t a = g0 + ng * qq / ns, z = g0 + ng * (qq + 1) / ns;
                gsubs.push_back(make_int4((int)a, (int)(z - a), (int)bi, 0));
            }
            g0 = g1;
        }
    }
    p->ngsub = (int64_t)gsubs.size();

    // ---------------- FP64 plans: kernel values phi((q - frac_a) / (w/2)) per node, axis and
    // cell, in FP64.  FP32 plans: per node the packed origin and u_a = frac_a - (w/2 - 1) in
    // (0, 1] as floats; the kernels evaluate phi from u_a
    const int dw = d * w;
    std::vector<double> kerv(p->prec == NLINT_FP64 ? (size_t)Mh * dw : 0);
    std::vector<int4> posv(p->prec == NLINT_FP32 ? (size_t)Mh : 0);
    if (p->prec == NLINT_FP32) {
        // u = 1 exactly iff frac_a = w/2 exactly, where the first cell's value is 0 (|z| = 1);
        // every other offset is kept below 1 in FP32 as well, so that its first cell keeps the
        // value next to the edge, exp(-beta), as in FP64
        const double off = 0.5 * w - 1.0;
        const float below1 = std::nextafter(1.0f, 0.0f);
        for (int64_t o = 0; o < Mh; o++) {
            float u[3] = {0.0f, 0.0f, 0.0f};
            for (int ax = 0; ax < d; ax++) {
                const double fr = frs[(size_t)ax * Mh + o];
                u[ax] = fr == 0.5 * w ? 1.0f : std::min((float)(fr - off), below1);
            }
            int4 r;
            r.x = rel[o];
            std::memcpy(&r.y, &u[0], 4);
            std::memcpy(&r.z, &u[1], 4);
            std::memcpy(&r.w, &u[2], 4);
            posv[o] = r;
        }
    } else {
        const double beta = p->beta, inv_half = 2.0 / w;
        auto work = [&](int64_t a0, int64_t a1) {
            for (int64_t o = a0; o < a1; o++)
                for (int ax = 0; ax < d; ax++) {
                    const double fr = frs[(size_t)ax * Mh + o];
                    for (int q = 0; q < w; q++) {
                        const double z = (q - fr) * inv_half, s2 = 1.0 - z * z;
                        kerv[(size_t)o * dw + ax * w + q] = s2 > 0.0 ? std::exp(beta * (std::sqrt(s2) - 1.0)) : 0.0;
                    }
                }
        };
        const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> th;
        for (int t = 0; t < nt; t++) th.emplace_back(work, Mh * t / nt, Mh * (t + 1) / nt);
        for (auto &t : th) t.join();
    }

    // ---------------- deconvolution factors f[m'] = (2 pi / n) / psi_hat(m), m = m' - N/2
    std::vector<double> qx, qw;
    gauss_legendre(256, qx, qw);
    const double alpha = (double)w * M_PI / (double)n;
    std::vector<double> fac(p->N);
    for (int64_t a = 0; a < p->N; a++) {
        const double m = (double)(a - p->N / 2);
        const double psi = alpha * es_ft(m * alpha, p->beta, qx, qw);
        fac[a] = (2.0 * M_PI / (double)n) / psi;
    }
    // twiddles exp(-2 pi i q / n), interleaved
    std::vector<double> tw(2 * (size_t)n);
    for (int qq = 0; qq < n; qq++) {
        tw[2 * qq] = std::cos(2.0 * M_PI * qq / n);
        tw[2 * qq + 1] = -std::sin(2.0 * M_PI * qq / n);
    }

    // ---------------- upload
    size_t acc = 0;
    int rc;
    if (p->prec == NLINT_FP64) {  // FP32 plans carry the origins in their node records
        CK(cudaMalloc((void **)&p->d_rel, rel.size() * sizeof(int32_t) + 4));
        CK(cudaMemcpy(p->d_rel, rel.data(), rel.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    CK(cudaMalloc((void **)&p->d_perm, perm.size() * sizeof(int32_t) + 4));
    CK(cudaMemcpy(p->d_perm, perm.data(), perm.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMalloc((void **)&p->d_mirror, mirror.size() * sizeof(int32_t) + 4));
    CK(cudaMemcpy(p->d_mirror, mirror.data(), mirror.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    acc += ((p->prec == NLINT_FP64 ? rel.size() : 0) + perm.size() + mirror.size()) * 4;
    CK(cudaMalloc((void **)&p->d_subs, sizeof(int4) * std::max<size_t>(subs.size(), 1)));
    if (!subs.empty()) CK(cudaMemcpy(p->d_subs, subs.data(), sizeof(int4) * subs.size(), cudaMemcpyHostToDevice));
    if (grouped) {
        CK(cudaMalloc((void **)&p->d_gsubs, sizeof(int4) * std::max<size_t>(gsubs.size(), 1)));
        if (!gsubs.empty())
            CK(cudaMemcpy(p->d_gsubs, gsubs.data(), sizeof(int4) * gsubs.size(), cudaMemcpyHostToDevice));
        CK(cudaMalloc((void **)&p->d_grp, sizeof(int32_t) * grp.size()));
        CK(cudaMemcpy(p->d_grp, grp.data(), sizeof(int32_t) * grp.size(), cudaMemcpyHostToDevice));
        acc += sizeof(int4) * gsubs.size() + sizeof(int32_t) * grp.size();
    }
    CK(cudaMalloc((void **)&p->d_bins, sizeof(int4) * std::max<size_t>(bins.size(), 1)));
    if (!bins.empty()) CK(cudaMemcpy(p->d_bins, bins.data(), sizeof(int4) * bins.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc((void **)&p->d_crowd_bin, sizeof(int32_t) * std::max<size_t>(crowd_bin.size(), 1)));
    if (!crowd_bin.empty())
        CK(cudaMemcpy(p->d_crowd_bin, crowd_bin.data(), sizeof(int32_t) * crowd_bin.size(), cudaMemcpyHostToDevice));
    acc += sizeof(int4) * (subs.size() + bins.size()) + 4 * crowd_bin.size();
    {
        const int row = tile_pitch(p->prec == NLINT_FP64, d, w, p->bin_shape);
        // FP32 tiles have 4-byte cells (32 banks, one wavefront per warp), FP64 tiles 8-byte
        // cells (16 banks per half-warp wavefront); both kernels read / add one plane at a time
        const int L = node_lanes(w);
        const std::vector<int16_t> po = p->prec == NLINT_FP32 ? build_pair_order(w, row, 32, L, 32)
                                                              : build_pair_order(w, row, 16, L, 16);
        const std::vector<int16_t> &pi = po;
        CK(cudaMalloc((void **)&p->d_pairs, po.size() * sizeof(int16_t)));
        CK(cudaMemcpy(p->d_pairs, po.data(), po.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
        CK(cudaMalloc((void **)&p->d_pairs_i, pi.size() * sizeof(int16_t)));
        CK(cudaMemcpy(p->d_pairs_i, pi.data(), pi.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
        acc += po.size() * sizeof(int16_t);
    }

    {
        int64_t cells = 1;
        for (int ax = 0; ax < d; ax++) cells *= p->T[ax];
        p->bytes_crowd = sizeof(double2) * (size_t)cells * (size_t)p->ncrowd;
        if (p->bytes_crowd) {
            CK(cudaMalloc((void **)&p->d_crowd, p->bytes_crowd));
            acc += p->bytes_crowd;
        }
    }
    if (p->prec == NLINT_FP32) {
        CK(cudaMalloc((void **)&p->d_pos, sizeof(int4) * std::max<size_t>(posv.size(), 1)));
        if (!posv.empty())
            CK(cudaMemcpy(p->d_pos, posv.data(), sizeof(int4) * posv.size(), cudaMemcpyHostToDevice));
        acc += sizeof(int4) * posv.size();
        if ((rc = upload<float>(&p->d_W, Ws, acc))) return rc;
        if ((rc = upload<float>(&p->d_fac, fac, acc))) return rc;
        if ((rc = upload<float>(&p->d_tw, tw, acc))) return rc;
    } else {
        if ((rc = upload<double>(&p->d_ker, kerv, acc))) return rc;
        if ((rc = upload<double>(&p->d_W, Ws, acc))) return rc;
        if ((rc = upload<double>(&p->d_fac, fac, acc))) return rc;
        if ((rc = upload<double>(&p->d_tw, tw, acc))) return rc;
    }

    // ---------------- pass descriptors and workspaces
    const int64_t N = p->N, nh = n / 2 + 1;
    const size_t cs = p->prec == NLINT_FP32 ? 8 : 16;
    auto base = [&](PassDesc &pd, int sign) {
        std::memset(&pd, 0, sizeof(pd));
        pd.n = n;
        make_radix(n, pd);
        pd.sign = sign;
        pd.N = (int)N;
        pd.dim = d;
        pd.fac = p->d_fac;
    };
    if (d == 3) {
        base(p->P1, -1);
        p->P1.in_kind = IN_REAL_MODES; p->P1.out_kind = OUT_CPLX_HALF;
        p->P1.I = N * N; p->P1.n_outer = 1; p->P1.in_sa = N * N; p->P1.out_sa = N * N;
        base(p->P2, -1);
        p->P2.in_kind = IN_CPLX_MODES; p->P2.out_kind = OUT_CPLX_FULL;
        p->P2.I = N; p->P2.n_outer = nh; p->P2.in_so = N * N; p->P2.in_sa = N;
        p->P2.out_so = (int64_t)n * N; p->P2.out_sa = N;
        base(p->P3, -1);
        p->P3.in_kind = IN_CPLX_MODES; p->P3.out_kind = OUT_CPLX_FULL;
        p->P3.I = nh * n; p->P3.in_so = N; p->P3.out_so = n;
        base(p->Q1, +1);
        p->Q1.in_kind = IN_CPLX_FOLD; p->Q1.out_kind = OUT_CPLX_MODES;
        p->Q1.I = nh * n; p->Q1.out_so = N; p->Q1.fold_pad = p->pad;
        p->Q1.fold_plane = (int64_t)n * n; p->Q1.fold_rows_per_plane = n;
        base(p->Q2, +1);
        p->Q2.in_kind = IN_CPLX_FULL; p->Q2.out_kind = OUT_CPLX_MODES;
        p->Q2.I = N; p->Q2.n_outer = nh; p->Q2.in_so = (int64_t)n * N; p->Q2.in_sa = N;
        p->Q2.out_so = N * N; p->Q2.out_sa = N;
        base(p->Q3, +1);
        p->Q3.in_kind = IN_CPLX_HERM; p->Q3.out_kind = OUT_REAL_MODES;
        p->Q3.I = N * N; p->Q3.n_outer = 1; p->Q3.in_sa = N * N; p->Q3.out_sa = N * N;
        p->bytes_A = (size_t)nh * N * N * cs;
        p->bytes_B = (size_t)nh * n * N * cs;
        p->bytes_G = (size_t)nh * n * n * cs;
        p->bytes_Hext = (size_t)(nh + 2 * p->pad) * n * n * cs;
    } else {
        base(p->P1, -1);
        p->P1.in_kind = IN_REAL_MODES; p->P1.out_kind = OUT_CPLX_HALF;
        p->P1.I = N; p->P1.n_outer = 1; p->P1.in_sa = N; p->P1.out_sa = N;
        base(p->P3, -1);
        p->P3.in_kind = IN_CPLX_MODES; p->P3.out_kind = OUT_CPLX_FULL;
        p->P3.I = nh; p->P3.in_so = N; p->P3.out_so = n;
        base(p->Q1, +1);
        p->Q1.in_kind = IN_CPLX_FOLD; p->Q1.out_kind = OUT_CPLX_MODES;
        p->Q1.I = nh; p->Q1.out_so = N; p->Q1.fold_pad = p->pad;
        p->Q1.fold_plane = n; p->Q1.fold_rows_per_plane = 1;
        base(p->Q3, +1);
        p->Q3.in_kind = IN_CPLX_HERM; p->Q3.out_kind = OUT_REAL_MODES;
        p->Q3.I = N; p->Q3.n_outer = 1; p->Q3.in_sa = N; p->Q3.out_sa = N;
        p->bytes_A = (size_t)nh * N * cs;
        p->bytes_B = 0;
        p->bytes_G = (size_t)nh * n * cs;
        p->bytes_Hext = (size_t)(nh + 2 * p->pad) * n * cs;
    }
    if (p->P1.nrad < 0) return fail(NLINT_EUNSUPPORTED, "fine grid size is not 2^a 3^b");
    p->P3.ball2 = p->Q1.ball2 = p->ball2;
    config_pass(p->P1, p->prec, false, p->fft_sched);
    config_pass(p->P3, p->prec, true, p->fft_sched);
    config_pass(p->Q1, p->prec, true, p->fft_sched);
    config_pass(p->Q3, p->prec, false, p->fft_sched);
    if (d == 3) {
        config_pass(p->P2, p->prec, false, p->fft_sched);
        config_pass(p->Q2, p->prec, false, p->fft_sched);
    }
    for (PassDesc *pd : {&p->P1, &p->P3, &p->Q1, &p->Q3})
        if (!pass_fits(*pd)) return fail(NLINT_EUNSUPPORTED, "internal: FFT pass does not fit");
    if (d == 3 && (!pass_fits(p->P2) || !pass_fits(p->Q2)))
        return fail(NLINT_EUNSUPPORTED, "internal: FFT pass does not fit");
    p->n_partials = (int)pass_blocks(p->Q3, false);
    p->bytes_c = (size_t)Mh * cs;
    CK(cudaMalloc(&p->d_bufA, p->bytes_A));
    if (p->bytes_B) CK(cudaMalloc(&p->d_bufB, p->bytes_B));
    CK(cudaMalloc(&p->d_bufG, std::max(p->bytes_G, p->bytes_Hext)));
    CK(cudaMalloc(&p->d_c, p->bytes_c + cs));
    // + 64: scratch of the two-stage energy fold (launch_energy_final)
    CK(cudaMalloc((void **)&p->d_partials, sizeof(double2) * ((size_t)std::max(p->n_partials, 1024) + 64)));
    CK(cudaMalloc((void **)&p->d_epart,
                  sizeof(double2) * ((size_t)std::max<int64_t>(std::max(p->nsub, p->ngsub), 1) + 64)));
    acc += sizeof(double2) * (size_t)std::max(p->nsub, p->ngsub);
    CK(cudaMalloc((void **)&p->d_E, sizeof(double)));
    acc += p->bytes_A + p->bytes_B + std::max(p->bytes_G, p->bytes_Hext) + p->bytes_c +
           sizeof(double2) * (size_t)std::max(p->n_partials, 1024);
    if (p->algorithm == 1) {
        // a separate spread grid when memory allows (else the spreading reuses d_bufG)
        if (cudaMalloc(&p->d_bufH, p->bytes_Hext) == cudaSuccess) {
            CK(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&p->ev_zero, cudaEventDisableTiming));
            acc += p->bytes_Hext;
        } else {
            (void)cudaGetLastError();
            p->d_bufH = nullptr;
        }
    }
    // FP32 3D Algorithm 1: a tensor map of the fine grid (the stored half, 8-byte cells) for the
    // interpolation's TMA tile loads; without one the kernels stage tiles by plain loads
    CK(cudaMalloc((void **)&p->d_status, sizeof(int)));
    CK(cudaMemset(p->d_status, 0, sizeof(int)));
    if (p->prec == NLINT_FP32 && d == 3 && p->algorithm == 1 && p->ngsub > 0)
        p->has_tmap = encode_grid_tmap(&p->tmapG, p->d_bufG, n, p->T);
    p->ws_bytes = acc;
    if (p->algorithm == 2) return alg2_setup(p);
    return NLINT_OK;
}

// ------------------------------------------------------------------------- FFT convolution
// Unit deconvolution factors for the passes of an FFT convolution on the fine grid.
static int upload_ones(nlint_plan_s *p) {
    if (p->d_fac1) return NLINT_OK;
    std::vector<double> ones((size_t)std::max<int64_t>(p->N, p->n_fine), 1.0);
    size_t acc = 0;
    return p->prec == NLINT_FP32 ? upload<float>(&p->d_fac1, ones, acc) : upload<double>(&p->d_fac1, ones, acc);
}

// Passes of u = crop(IFFT(K_hat FFT(rho_pad))) on the fine grid: the NUFFT passes with unit
// factors along z and y, and one row pass along x that transforms each line forward, multiplies
// it by its row of the real half grid d_khat and transforms it back (the spectrum never goes to
// memory).
static void conv_passes(nlint_plan_s *p) {
    const int d = p->d, n = p->n_fine;
    const int64_t N = p->N, nh = n / 2 + 1;
    p->T1 = p->P1;
    p->T1.fac = p->d_fac1;
    p->U3 = p->Q3;
    p->U3.fac = p->d_fac1;
    std::memset(&p->X, 0, sizeof(p->X));
    p->X.n = n;
    make_radix(n, p->X);
    p->X.sign = -1;
    p->X.N = (int)N;
    p->X.dim = d;
    p->X.in_kind = IN_CPLX_MODES;
    p->X.out_kind = OUT_CPLX_MODES;
    p->X.I = (d == 3) ? nh * n : nh;
    p->X.in_so = N;
    p->X.out_so = N;
    p->X.mult = p->d_khat;
    p->X.conv = 1;
    config_pass(p->X, p->prec, true, p->fft_sched);
}

// Algorithm 2: I_1's multiplier M(k) / n_fine^d on the real half grid of the fine grid's DFT
// (axis 0 non-negative frequencies 0..n/2, the others in FFT order; frequency index g <-> k =
// 2 pi g' / (n_fine h) with g' the signed index, n/2 -> -n/2), in the plan precision.
template <typename T>
static int alg2_fill_multiplier(nlint_plan_s *p) {
    const int d = p->d, n = p->n_fine;
    const int64_t nh = n / 2 + 1, rows = (d == 3) ? nh * n : nh;
    const double dk = 2.0 * M_PI / ((double)n * p->h);
    const double inv = 1.0 / std::pow((double)n, d);
    std::vector<T> m((size_t)(rows * n));
    std::vector<int64_t> row_r2(rows, -1);  // s0^2 + s1^2 of each row with a nonzero entry
    auto sgn = [n](int64_t g) { return (double)(g < n / 2 ? g : g - n); };
    auto work = [&](int64_t r0, int64_t r1) {
        for (int64_t r = r0; r < r1; r++) {
            const int64_t g0 = (d == 3) ? r / n : r, g1 = (d == 3) ? r % n : 0;
            for (int64_t c = 0; c < n; c++) {
                double k[3] = {0.0, 0.0, 0.0};
                if (d == 3) {
                    k[2] = dk * sgn(g0);  // array axis 0 is z
                    k[1] = dk * sgn(g1);
                    k[0] = dk * sgn(c);
                } else {
                    k[1] = dk * sgn(g0);  // array axis 0 is y
                    k[0] = dk * sgn(c);
                }
                m[(size_t)(r * n + c)] = (T)(alg2_multiplier(p, k) * inv);
                if (m[(size_t)(r * n + c)] != T(0)) {
                    const int64_t s0 = (d == 3) ? (int64_t)sgn(g0) : g0, s1 = (d == 3) ? (int64_t)sgn(g1) : 0;
                    row_r2[r] = s0 * s0 + s1 * s1;
                }
            }
        }
    };
    const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (int t = 0; t < nt; t++) th.emplace_back(work, rows * t / nt, rows * (t + 1) / nt);
    for (auto &t : th) t.join();
    // the convolution pass skips the rows beyond every nonzero multiplier row (PassDesc::ball2)
    int64_t r2max = 0;
    for (int64_t v : row_r2) r2max = std::max(r2max, v);
    const int64_t full = (d == 3) ? 2 * (int64_t)(n / 2) * (n / 2) : (int64_t)(n / 2) * (n / 2);
    p->conv_ball2 = r2max < full ? std::max<int64_t>(r2max, 1) : 0;
    CK(cudaMalloc(&p->d_khat, m.size() * sizeof(T)));
    CK(cudaMemcpy(p->d_khat, m.data(), m.size() * sizeof(T), cudaMemcpyHostToDevice));
    p->ws_bytes += m.size() * sizeof(T);
    return NLINT_OK;
}

// I_2's windowed passes: the nodes of I_2 lie within |k| <= P2, so with t = k h their stencils
// cover fine cells |l| <= P2 h n / (2 pi) + w/2 + 1 on every axis.  The forward passes compute
// only those frequencies (the last one writes them at their place in the fine grid, where the
// interpolation reads them), and the inverse passes transform only those lines of the spread
// grid.  Needs the window well inside the half grid (no fold at the Nyquist planes).
static void alg2_window(nlint_plan_s *p) {
    const int d = p->d, n = p->n_fine;
    const int64_t N = p->N;
    const double g = p->rad2 * p->h * (double)n / (2.0 * M_PI);
    const int win = (int)std::ceil(g) + p->w / 2 + 2;
    if (win + p->pad + 1 >= n / 2 - p->pad || 2 * win + 1 > n) return;  // window too wide
    const int wr = 2 * win + 1;
    const size_t cs = p->prec == NLINT_FP32 ? 8 : 16;
    auto base = [&](PassDesc &pd, int sign, int in_kind, int out_kind) {
        std::memset(&pd, 0, sizeof(pd));
        pd.n = n;
        make_radix(n, pd);
        pd.sign = sign;
        pd.N = (int)N;
        pd.dim = d;
        pd.fac = p->d_fac;
        pd.in_kind = in_kind;
        pd.out_kind = out_kind;
        pd.win = win;
    };
    if (d == 3) {
        base(p->P1w, -1, IN_REAL_MODES, OUT_CPLX_HALF);
        p->P1w.I = N * N; p->P1w.n_outer = 1; p->P1w.in_sa = N * N; p->P1w.out_sa = N * N;
        base(p->P2w, -1, IN_CPLX_MODES, OUT_CPLX_WIN);
        p->P2w.I = N; p->P2w.n_outer = win + 1; p->P2w.in_so = N * N; p->P2w.in_sa = N;
        p->P2w.out_so = (int64_t)wr * N; p->P2w.out_sa = N;
        base(p->P3w, -1, IN_CPLX_MODES, OUT_CPLX_FULL);
        p->P3w.I = (int64_t)(win + 1) * wr; p->P3w.in_so = N; p->P3w.out_so = n; p->P3w.win_rows = wr;
        base(p->Q1w, +1, IN_CPLX_FOLD, OUT_CPLX_MODES);
        p->Q1w.I = (int64_t)(win + 1) * wr; p->Q1w.out_so = N; p->Q1w.fold_pad = p->pad;
        p->Q1w.fold_plane = (int64_t)n * n; p->Q1w.fold_rows_per_plane = n; p->Q1w.win_rows = wr;
        base(p->Q2w, +1, IN_CPLX_WIN, OUT_CPLX_MODES);
        p->Q2w.I = N; p->Q2w.n_outer = win + 1; p->Q2w.in_so = (int64_t)wr * N; p->Q2w.in_sa = N;
        p->Q2w.out_so = N * N; p->Q2w.out_sa = N;
        base(p->Q3w, +1, IN_CPLX_HERM, OUT_REAL_MODES);
        p->Q3w.I = N * N; p->Q3w.n_outer = 1; p->Q3w.in_sa = N * N; p->Q3w.out_sa = N * N;
        config_pass(p->P2w, p->prec, false, p->fft_sched);
        config_pass(p->P3w, p->prec, true, p->fft_sched);
        config_pass(p->Q2w, p->prec, false, p->fft_sched);
        p->bytes_Hwin = (size_t)(win + 2 * p->pad + 1) * n * n * cs;
    } else {
        base(p->P1w, -1, IN_REAL_MODES, OUT_CPLX_HALF);
        p->P1w.I = N; p->P1w.n_outer = 1; p->P1w.in_sa = N; p->P1w.out_sa = N;
        base(p->P3w, -1, IN_CPLX_MODES, OUT_CPLX_FULL);
        p->P3w.I = win + 1; p->P3w.in_so = N; p->P3w.out_so = n;
        base(p->Q1w, +1, IN_CPLX_FOLD, OUT_CPLX_MODES);
        p->Q1w.I = win + 1; p->Q1w.out_so = N; p->Q1w.fold_pad = p->pad;
        p->Q1w.fold_plane = n; p->Q1w.fold_rows_per_plane = 1;
        base(p->Q3w, +1, IN_CPLX_HERM, OUT_REAL_MODES);
        p->Q3w.I = N; p->Q3w.n_outer = 1; p->Q3w.in_sa = N; p->Q3w.out_sa = N;
        config_pass(p->P3w, p->prec, true, p->fft_sched);
        p->bytes_Hwin = (size_t)(win + 2 * p->pad + 1) * n * cs;
    }
    config_pass(p->P1w, p->prec, false, p->fft_sched);
    config_pass(p->Q1w, p->prec, true, p->fft_sched);
    config_pass(p->Q3w, p->prec, false, p->fft_sched);
    if (pass_blocks(p->Q3w, false) > p->n_partials) return;  // (same grid as Q3: never)
    p->win = win;
    // the dual z passes (I_1 with unit factors, I_2 with the deconvolution) when their grid fits
    // the energy partials
    auto dual = [&](PassDesc &dst, const PassDesc &src) {
        dst = src;
        dst.dual = 1;
        dst.fac = p->d_fac1;
        dst.fac2 = p->d_fac;
        config_pass(dst, p->prec, false, p->fft_sched);
    };
    dual(p->D6, p->P1w);
    dual(p->D7, p->Q3w);
    p->bytes_win = (size_t)(win + 1) * (d == 3 ? N * N : N) * cs;
    p->dual = pass_fits(p->D6) && pass_fits(p->D7) && pass_blocks(p->D7, false) <= p->n_partials;
}

static int alg2_setup(nlint_plan_s *p) {
    int rc = upload_ones(p);
    if (rc) return rc;
    alg2_window(p);
    if (p->win > 0 && p->dual) {
        CK(cudaMalloc(&p->d_win, p->bytes_win));
        p->ws_bytes += p->bytes_win;
    }
    p->ws_bytes += (size_t)std::max<int64_t>(p->N, p->n_fine) * (p->prec == NLINT_FP32 ? 4 : 8);
    rc = p->prec == NLINT_FP32 ? alg2_fill_multiplier<float>(p) : alg2_fill_multiplier<double>(p);
    if (rc) return rc;
    conv_passes(p);
    p->X.ball2 = p->conv_ball2;
    return NLINT_OK;
}

// ------------------------------------------------------------------------- execution
static void stage_mark(nlint_plan_s *p, cudaStream_t s, const char *name) {
    if (!p->timing) return;
    if (p->ev_used >= (int)p->ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        p->ev.push_back(e);
        p->ev_names.push_back(name);
    }
    p->ev_names[p->ev_used] = name;
    cudaEventRecord(p->ev[p->ev_used], s);
    p->ev_used++;
}

template <typename T>
static int run_type2(nlint_plan_s *p, const void *rho, cudaStream_t s) {
    CK(launch_colpass<T>(p->P1, rho, p->d_bufA, p->d_tw, s));
    p->launches += (p->d == 3) ? 3 : 2;
    if (p->d == 3) {
        stage_mark(p, s, "fwd_fft_z");
        CK(launch_colpass<T>(p->P2, p->d_bufA, p->d_bufB, p->d_tw, s));
        stage_mark(p, s, "fwd_fft_y");
        CK(launch_rowpass<T>(p->P3, p->d_bufB, p->d_bufG, p->d_tw, s));
        stage_mark(p, s, "fwd_fft_x");
    } else {
        stage_mark(p, s, "fwd_fft_y");
        CK(launch_rowpass<T>(p->P3, p->d_bufA, p->d_bufG, p->d_tw, s));
        stage_mark(p, s, "fwd_fft_x");
    }
    return NLINT_OK;
}

// Stencil values of the FP32 3D interpolation as polynomials (the piecewise-polynomial kernel
// evaluation of Barnett, Magland and af Klinteberg): on stencil cell q the value
// phi(z), z = (q + 1 - w/2) (2/w) - u (2/w) for the node offset u in [0, 1], is interpolated at
// the D + 1 Chebyshev points of t = 2u - 1 in [-1, 1] (FP64), and the Chebyshev series turned
// into monomial coefficients in t.  The fit is kept only if FP32 Horner evaluation by fused
// multiply-adds stays within 1.5e-7 of phi (absolute; phi <= 1) on a fine grid of u; else the
// kernels evaluate phi by its formula.
static void fit_phi_poly(nlint_plan_s *p) {
    p->phpoly = 0;
    const int w = p->w;
    if (p->prec != NLINT_FP32 || p->d != 3 || w < 7 || w > NODE_MAXW) return;
    const int D = ph_degree(w), NC = D + 1;
    const double beta = p->beta;
    auto phi = [&](double z) {
        const double t = 1.0 - z * z;
        return t > 0.0 ? std::exp(-beta * z * z / (1.0 + std::sqrt(t))) : std::exp(-beta);
    };
    float coef[NODE_MAXW * PH_NC] = {};
    for (int q = 0; q < w; q++) {
        const double vc = (q + 1.0 - 0.5 * w) * (2.0 / w);
        double val[PH_NC], cheb[PH_NC];
        for (int k = 0; k < NC; k++) {
            const double tk = std::cos(M_PI * (k + 0.5) / NC);
            val[k] = phi(vc - (tk + 1.0) / w);
        }
        for (int j = 0; j < NC; j++) {
            double a = 0.0;
            for (int k = 0; k < NC; k++) a += val[k] * std::cos(j * M_PI * (k + 0.5) / NC);
            cheb[j] = a * (j == 0 ? 1.0 : 2.0) / NC;
        }
        // monomials: T_0 = 1, T_1 = t, T_{j+1} = 2 t T_j - T_{j-1}, as coefficient vectors
        double mono[PH_NC] = {}, Tm[PH_NC] = {}, T0[PH_NC] = {}, T1[PH_NC] = {};
        T0[0] = 1.0;
        T1[1] = 1.0;
        for (int j = 0; j < NC; j++) {
            const double *Tj = j == 0 ? T0 : T1;
            for (int k = 0; k < NC; k++) mono[k] += cheb[j] * Tj[k];
            if (j >= 1) {  // advance: Tm = 2 t T1 - T0
                for (int k = 0; k < NC; k++) Tm[k] = (k > 0 ? 2.0 * T1[k - 1] : 0.0) - T0[k];
                for (int k = 0; k < NC; k++) {
                    T0[k] = T1[k];
                    T1[k] = Tm[k];
                }
            }
        }
        for (int k = 0; k < NC; k++) coef[q * PH_NC + k] = (float)mono[k];
        for (int i = 0; i <= 4000; i++) {  // FP32 Horner as the kernel evaluates it
            const double u = i / 4000.0;
            const float t = std::fmaf(2.0f, (float)u, -1.0f);
            float acc = coef[q * PH_NC + D];
            for (int k = D - 1; k >= 0; k--) acc = std::fmaf(acc, t, coef[q * PH_NC + k]);
            if (!(std::fabs((double)acc - phi(vc - u * (2.0 / w))) <= 1.5e-7)) return;
        }
    }
    std::memcpy(p->phc, coef, sizeof coef);
    p->phpoly = 1;
}

static NodeDesc node_desc(nlint_plan_s *p) {
    NodeDesc nd;
    nd.d = p->d;
    nd.M = p->Mh;
    nd.n = p->n_fine;
    nd.w = p->w;
    nd.pad = p->pad;
    nd.beta = p->beta;
    nd.bin_shape = p->bin_shape;
    nd.pos = p->d_pos;
    nd.rel = p->d_rel;
    nd.ker = p->d_ker;
    nd.W = p->d_W;
    for (int a = 0; a < 3; a++) {
        nd.B[a] = p->B[a];
        nd.T[a] = p->T[a];
    }
    nd.nsub = p->nsub;
    nd.subs = p->d_subs;
    nd.ngsub = p->ngsub;
    nd.gsubs = p->d_gsubs;
    nd.grp = p->d_grp;
    nd.tmap = p->has_tmap ? &p->tmapG : nullptr;
    nd.status = p->d_status;
    nd.bins = p->d_bins;
    nd.ncrowd = p->ncrowd;
    nd.crowd = p->d_crowd;
    nd.crowd_bin = p->d_crowd_bin;
    nd.pair_order = p->d_pairs;
    nd.pair_order_i = p->d_pairs_i;
    nd.phpoly = p->phpoly;
    std::memcpy(nd.phc, p->phc, sizeof nd.phc);
    return nd;
}

// Clears the separate spread grid (and the crowd tiles) on the plan's side stream, ordered after
// everything already on `s` (the previous evaluation's reads of the grid); run_type1 waits for it.
static int clear_spread_grid(nlint_plan_s *p, cudaStream_t s) {
    CK(cudaEventRecord(p->ev_fork, s));
    CK(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
    CK(cudaMemsetAsync(p->d_bufH, 0, p->bytes_Hext, p->side));
    if (p->ncrowd) CK(cudaMemsetAsync(p->d_crowd, 0, p->bytes_crowd, p->side));
    CK(cudaEventRecord(p->ev_zero, p->side));
    return NLINT_OK;
}

template <typename T>
static int run_type1(nlint_plan_s *p, void *u, const void *rho_energy, cudaStream_t s,
                     bool accumulate = false) {
    void *H = p->d_bufH ? p->d_bufH : p->d_bufG;
    if (p->d_bufH) {
        CK(cudaStreamWaitEvent(s, p->ev_zero, 0));  // cleared by clear_spread_grid
    } else {
        CK(cudaMemsetAsync(H, 0, p->bytes_Hext, s));
        if (p->ncrowd) CK(cudaMemsetAsync(p->d_crowd, 0, p->bytes_crowd, s));
    }
    CK(launch_spread<T>(node_desc(p), p->d_c, H, s));
    if (p->ncrowd) {
        CK(launch_crowd_merge<T>(node_desc(p), H, s));
        p->launches += 1;
    }
    p->launches += (p->d == 3) ? 4 : 3;
    stage_mark(p, s, "spread");
    if (p->d == 3) {
        CK(launch_rowpass<T>(p->Q1, H, p->d_bufB, p->d_tw, s));
        stage_mark(p, s, "inv_fft_x");
        CK(launch_colpass<T>(p->Q2, p->d_bufB, p->d_bufA, p->d_tw, s));
        stage_mark(p, s, "inv_fft_y");
    } else {
        CK(launch_rowpass<T>(p->Q1, H, p->d_bufA, p->d_tw, s));
        stage_mark(p, s, "inv_fft_x");
    }
    PassDesc q3 = p->Q3;
    q3.rho = rho_energy;
    q3.partials = rho_energy ? p->d_partials : nullptr;
    q3.accum = accumulate ? 1 : 0;  // u += (Algorithm 2: I_2 onto I_1)
    CK(launch_colpass<T>(q3, p->d_bufA, u, p->d_tw, s));
    stage_mark(p, s, p->d == 3 ? "inv_fft_z" : "inv_fft_y");
    return NLINT_OK;
}

template <typename T>
static int run_alg2(nlint_plan_s *p, const void *rho, void *u, double lambda, double *E,
                    cudaStream_t s);

template <typename T>
static int run_eval(nlint_plan_s *p, const void *rho, void *u, double lambda, double *E,
                    cudaStream_t s) {
    if (p->algorithm == 2) return run_alg2<T>(p, rho, u, lambda, E, s);
    p->ev_used = 0;
    stage_mark(p, s, "start");
    int rc = run_type2<T>(p, rho, s);
    if (rc) return rc;
    if (p->d_bufH && (rc = clear_spread_grid(p, s))) return rc;  // overlaps the interpolation
    CK(launch_interp<T>(node_desc(p), p->d_bufG, p->d_c, 1, s));
    p->launches += 1;
    stage_mark(p, s, "interp");
    rc = run_type1<T>(p, u, E ? rho : nullptr, s);
    if (rc) return rc;
    if (E) {
        CK(launch_energy_final(p->d_partials, p->n_partials, 0.5 * lambda * std::pow(p->h, p->d), E, s));
        p->launches += energy_final_kernels(p->n_partials);
        stage_mark(p, s, "energy");
    }
    return NLINT_OK;
}

template <typename T>
static int run_toeplitz(nlint_plan_s *p, const void *rho, void *u, double lambda, double *E,
                        cudaStream_t s) {
    p->ev_used = 0;
    stage_mark(p, s, "start");
    CK(launch_colpass<T>(p->T1, rho, p->d_bufA, p->d_tw, s));
    if (p->d == 3) {
        CK(launch_colpass<T>(p->P2, p->d_bufA, p->d_bufB, p->d_tw, s));
        CK(launch_rowpass<T>(p->X, p->d_bufB, p->d_bufG, p->d_tw, s));  // x: FFT, K_hat, IFFT
    } else {
        CK(launch_rowpass<T>(p->X, p->d_bufA, p->d_bufG, p->d_tw, s));
    }
    stage_mark(p, s, "fwd_fft_conv_x");
    PassDesc u3 = p->U3;
    u3.rho = E ? rho : nullptr;
    u3.partials = E ? p->d_partials : nullptr;
    if (p->d == 3) {
        CK(launch_colpass<T>(p->Q2, p->d_bufG, p->d_bufA, p->d_tw, s));
        CK(launch_colpass<T>(u3, p->d_bufA, u, p->d_tw, s));
    } else {
        CK(launch_colpass<T>(u3, p->d_bufG, u, p->d_tw, s));
    }
    stage_mark(p, s, "inv_fft");
    p->launches += (p->d == 3) ? 5 : 3;
    if (E) {
        CK(launch_energy_final(p->d_partials, p->n_partials, 0.5 * lambda * std::pow(p->h, p->d), E, s));
        p->launches += energy_final_kernels(p->n_partials);
        stage_mark(p, s, "energy");
    }
    return NLINT_OK;
}

// Algorithm 2 with I_2 on its frequency window and the z passes of both integrals shared: one
// forward z pass reads rho once and writes I_1's half grid (bufA) and I_2's window planes
// (d_win); I_2's remaining passes and the NUFFT run on the window, then I_1's y / x-convolution
// / y passes; one inverse z pass forms u = I_1 + I_2 and the energy products.
template <typename T>
static int run_alg2_dual(nlint_plan_s *p, const void *rho, void *u, double lambda, double *E,
                         cudaStream_t s) {
    PassDesc d6 = p->D6;
    d6.out2 = p->d_win;
    CK(launch_colpass<T>(d6, rho, p->d_bufA, p->d_tw, s));
    stage_mark(p, s, "dual_fwd_z");
    if (p->d == 3) {
        CK(launch_colpass<T>(p->P2w, p->d_win, p->d_bufB, p->d_tw, s));
        CK(launch_rowpass<T>(p->P3w, p->d_bufB, p->d_bufG, p->d_tw, s));
    } else {
        CK(launch_rowpass<T>(p->P3w, p->d_win, p->d_bufG, p->d_tw, s));
    }
    stage_mark(p, s, "I2_fwd_fft");
    CK(launch_interp<T>(node_desc(p), p->d_bufG, p->d_c, 1, s));
    stage_mark(p, s, "interp");
    CK(cudaMemsetAsync(p->d_bufG, 0, p->bytes_Hwin, s));
    if (p->ncrowd) CK(cudaMemsetAsync(p->d_crowd, 0, p->bytes_crowd, s));
    CK(launch_spread<T>(node_desc(p), p->d_c, p->d_bufG, s));
    if (p->ncrowd) {
        CK(launch_crowd_merge<T>(node_desc(p), p->d_bufG, s));
        p->launches += 1;
    }
    stage_mark(p, s, "spread");
    if (p->d == 3) {
        CK(launch_rowpass<T>(p->Q1w, p->d_bufG, p->d_bufB, p->d_tw, s));
        CK(launch_colpass<T>(p->Q2w, p->d_bufB, p->d_win, p->d_tw, s));
    } else {
        CK(launch_rowpass<T>(p->Q1w, p->d_bufG, p->d_win, p->d_tw, s));
    }
    stage_mark(p, s, "I2_inv_fft");
    const void *half1;  // I_1's inverse-transformed half grid, before the last z pass
    if (p->d == 3) {
        CK(launch_colpass<T>(p->P2, p->d_bufA, p->d_bufB, p->d_tw, s));
        CK(launch_rowpass<T>(p->X, p->d_bufB, p->d_bufG, p->d_tw, s));  // x: FFT, M, IFFT
        CK(launch_colpass<T>(p->Q2, p->d_bufG, p->d_bufA, p->d_tw, s));
        half1 = p->d_bufA;
    } else {
        CK(launch_rowpass<T>(p->X, p->d_bufA, p->d_bufG, p->d_tw, s));
        half1 = p->d_bufG;
    }
    stage_mark(p, s, "I1_fft_conv");
    PassDesc d7 = p->D7;
    d7.in2 = p->d_win;
    d7.rho = E ? rho : nullptr;
    d7.partials = E ? p->d_partials : nullptr;
    CK(launch_colpass<T>(d7, half1, u, p->d_tw, s));
    stage_mark(p, s, "dual_inv_z");
    p->launches += (p->d == 3) ? 11 : 7;
    if (E) {
        CK(launch_energy_final(p->d_partials, p->n_partials, 0.5 * lambda * std::pow(p->h, p->d), E, s));
        p->launches += energy_final_kernels(p->n_partials);
        stage_mark(p, s, "energy");
    }
    return NLINT_OK;
}

// Algorithm 2 (Section 3.3, eq. 3.9): u = I_1 + I_2.  I_1 (step 3): zero-padded forward FFT of
// rho on the fine grid, multiply by U_hat (1 - p) (between the forward and inverse x transforms
// of one row pass), inverse FFT, crop -> u.  I_2 (step 4): the NUFFT path on I_2's nodes (weights W_j p(k_j)), its last
// pass adding onto u and taking the energy over the sum (step 5 and Remark 3.3).
template <typename T>
static int run_alg2(nlint_plan_s *p, const void *rho, void *u, double lambda, double *E,
                    cudaStream_t s) {
    p->ev_used = 0;
    stage_mark(p, s, "start");
    if (p->win > 0 && p->dual) return run_alg2_dual<T>(p, rho, u, lambda, E, s);
    CK(launch_colpass<T>(p->T1, rho, p->d_bufA, p->d_tw, s));
    if (p->d == 3) {
        CK(launch_colpass<T>(p->P2, p->d_bufA, p->d_bufB, p->d_tw, s));
        CK(launch_rowpass<T>(p->X, p->d_bufB, p->d_bufG, p->d_tw, s));  // x: FFT, M, IFFT
        CK(launch_colpass<T>(p->Q2, p->d_bufG, p->d_bufA, p->d_tw, s));
        CK(launch_colpass<T>(p->U3, p->d_bufA, u, p->d_tw, s));
    } else {
        CK(launch_rowpass<T>(p->X, p->d_bufA, p->d_bufG, p->d_tw, s));
        CK(launch_colpass<T>(p->U3, p->d_bufG, u, p->d_tw, s));
    }
    p->launches += (p->d == 3) ? 5 : 3;
    stage_mark(p, s, "I1_fft_conv");
    if (p->win > 0) {
        // I_2 on its frequency window
        CK(launch_colpass<T>(p->P1w, rho, p->d_bufA, p->d_tw, s));
        if (p->d == 3) {
            CK(launch_colpass<T>(p->P2w, p->d_bufA, p->d_bufB, p->d_tw, s));
            CK(launch_rowpass<T>(p->P3w, p->d_bufB, p->d_bufG, p->d_tw, s));
        } else {
            CK(launch_rowpass<T>(p->P3w, p->d_bufA, p->d_bufG, p->d_tw, s));
        }
        stage_mark(p, s, "I2_fwd_fft");
        CK(launch_interp<T>(node_desc(p), p->d_bufG, p->d_c, 1, s));
        stage_mark(p, s, "interp");
        CK(cudaMemsetAsync(p->d_bufG, 0, p->bytes_Hwin, s));
        if (p->ncrowd) CK(cudaMemsetAsync(p->d_crowd, 0, p->bytes_crowd, s));
        CK(launch_spread<T>(node_desc(p), p->d_c, p->d_bufG, s));
        if (p->ncrowd) {
            CK(launch_crowd_merge<T>(node_desc(p), p->d_bufG, s));
            p->launches += 1;
        }
        stage_mark(p, s, "spread");
        PassDesc q3 = p->Q3w;
        q3.rho = E ? rho : nullptr;
        q3.partials = E ? p->d_partials : nullptr;
        q3.accum = 1;
        if (p->d == 3) {
            CK(launch_rowpass<T>(p->Q1w, p->d_bufG, p->d_bufB, p->d_tw, s));
            CK(launch_colpass<T>(p->Q2w, p->d_bufB, p->d_bufA, p->d_tw, s));
        } else {
            CK(launch_rowpass<T>(p->Q1w, p->d_bufG, p->d_bufA, p->d_tw, s));
        }
        CK(launch_colpass<T>(q3, p->d_bufA, u, p->d_tw, s));
        stage_mark(p, s, "I2_inv_fft");
        p->launches += (p->d == 3) ? 8 : 6;
    } else {
        int rc = run_type2<T>(p, rho, s);
        if (rc) return rc;
        CK(launch_interp<T>(node_desc(p), p->d_bufG, p->d_c, 1, s));
        p->launches += 1;
        stage_mark(p, s, "interp");
        rc = run_type1<T>(p, u, E ? rho : nullptr, s, true);
        if (rc) return rc;
    }
    if (E) {
        CK(launch_energy_final(p->d_partials, p->n_partials, 0.5 * lambda * std::pow(p->h, p->d), E, s));
        p->launches += energy_final_kernels(p->n_partials);
        stage_mark(p, s, "energy");
    }
    return NLINT_OK;
}

static int check_plan(nlint_plan p) {
    if (!p) return fail(NLINT_EINVAL, "plan is NULL");
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return NLINT_OK;
}

}  // namespace nlint

using namespace nlint;

// =============================================================================== C-ABI
extern "C" {

void nlint_params_default(nlint_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->d = 3;
    p->n = 32;
    p->L = 16.0;
    p->kernel = NLINT_COULOMB;
    p->eps = 1e-6;
    p->precision = -1;
    p->device = -1;
    p->algorithm = 1;
}

int nlint_plan_create_ex(const nlint_params *prm, nlint_plan *out) {
    if (!prm || !out) return fail(NLINT_EINVAL, "NULL argument");
    *out = nullptr;
    nlint_plan_s *p = new (std::nothrow) nlint_plan_s();
    if (!p) return fail(NLINT_ENOMEM, "host allocation failed");
    int rc;
    try {
        rc = build_plan(prm, p);
    } catch (const std::bad_alloc &) {
        rc = fail(NLINT_ENOMEM, "host allocation failed");
    } catch (...) {
        rc = fail(NLINT_EINVAL, "unexpected error while building the plan");
    }
    if (rc != NLINT_OK) {
        plan_free(p);
        delete p;
        return rc;
    }
    g_err.clear();
    *out = p;
    return NLINT_OK;
}

int nlint_plan_create(int d, int64_t n, double L, int kernel, const double *dipole_axis,
                      double eps, nlint_plan *out) {
    nlint_params prm;
    nlint_params_default(&prm);
    prm.d = d;
    prm.n = n;
    prm.L = L;
    prm.kernel = kernel;
    prm.eps = eps;
    if (kernel == NLINT_DIPOLE) {
        if (!dipole_axis) return fail(NLINT_EINVAL, "dipole kernel needs an axis");
        for (int a = 0; a < 3; a++) prm.axis[a] = dipole_axis[a];
    }
    return nlint_plan_create_ex(&prm, out);
}

void nlint_plan_destroy(nlint_plan p) {
    if (!p) return;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    plan_free(p);
    delete p;
}

int nlint_plan_check(nlint_plan p) {
    if (!p) return fail(NLINT_EINVAL, "NULL plan");
    if (cudaSetDevice(p->device) != cudaSuccess) return fail(NLINT_ECUDA, "cudaSetDevice failed");
    int st = 0;
    if (cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(NLINT_ECUDA, "reading the plan's status word failed");
    if (st) {
        if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess)
            return fail(NLINT_ECUDA, "clearing the plan's status word failed");
        return fail(NLINT_ETIMEOUT, "a bounded device-side wait ran out (the results of that evaluation are invalid)");
    }
    return NLINT_OK;
}

int nlint_plan_info(nlint_plan p, nlint_info *info) {
    if (!p || !info) return fail(NLINT_EINVAL, "NULL argument");
    info->d = p->d;
    info->precision = p->prec;
    info->w = p->w;
    info->kernel = p->prm.kernel;
    info->n = p->N;
    info->n_fine = p->n_fine;
    info->n_nodes = p->Nf;
    info->n_half_nodes = p->Mh;
    info->n_r = p->nr;
    info->n_theta = p->d == 3 ? p->nt : 0;
    info->n_phi = p->nphi;
    info->L = p->L;
    info->h = p->h;
    info->P = p->P;
    info->sigma = (double)p->n_fine / (double)p->N;
    info->beta = p->beta;
    info->workspace_bytes = p->ws_bytes;
    info->n_bins = p->nbins;
    info->n_subproblems = p->nsub;
    info->n_crowd_bins = p->ncrowd;
    for (int a = 0; a < 3; a++) info->bin[a] = p->B[a];
    info->bin_shape = p->bin_shape;
    info->fft_sched = (int)p->fft_sched;
    info->device = p->device;
    info->algorithm = p->algorithm;
    info->pu_a = p->pu_a;
    info->pu_r0 = p->pu_r0;
    info->pu_r1 = p->pu_r1;
    info->P2 = p->rad2;
    info->toeplitz = p->toeplitz ? 1 : 0;
    return NLINT_OK;
}

int nlint_plan_nodes(nlint_plan p, double *k_host, double *W_host) {
    if (!p) return fail(NLINT_EINVAL, "plan is NULL");
    if (k_host) std::memcpy(k_host, p->k_canon.data(), p->k_canon.size() * sizeof(double));
    if (W_host) std::memcpy(W_host, p->W_canon.data(), p->W_canon.size() * sizeof(double));
    return NLINT_OK;
}

int nlint_eval(nlint_plan p, const void *rho, void *u, void *stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!rho || !u) return fail(NLINT_EINVAL, "NULL rho or u");
    cudaStream_t s = (cudaStream_t)stream;
    return p->prec == NLINT_FP32 ? run_eval<float>(p, rho, u, 0.0, nullptr, s)
                                 : run_eval<double>(p, rho, u, 0.0, nullptr, s);
}

int nlint_eval_energy(nlint_plan p, const void *rho, void *u, double lambda, double *E_dev,
                      void *stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!rho || !u) return fail(NLINT_EINVAL, "NULL rho or u");
    cudaStream_t s = (cudaStream_t)stream;
    double *E = E_dev ? E_dev : p->d_E;
    return p->prec == NLINT_FP32 ? run_eval<float>(p, rho, u, lambda, E, s)
                                 : run_eval<double>(p, rho, u, lambda, E, s);
}

int nlint_energy(nlint_plan p, const void *rho, const void *u, double lambda, double *E_dev,
                 double *E_host, void *stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!rho || !u) return fail(NLINT_EINVAL, "NULL rho or u");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t count = 1;
    for (int a = 0; a < p->d; a++) count *= p->N;
    const int nb = 1024;
    if (p->prec == NLINT_FP32) CK(launch_energy_partials<float>(count, u, rho, p->d_partials, nb, s));
    else CK(launch_energy_partials<double>(count, u, rho, p->d_partials, nb, s));
    double *E = E_dev ? E_dev : p->d_E;
    CK(launch_energy_final(p->d_partials, nb, 0.5 * lambda * std::pow(p->h, p->d), E, s));
    p->launches += 1 + energy_final_kernels(nb);
    if (E_host) {
        CK(cudaMemcpyAsync(E_host, E, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return NLINT_OK;
}

int nlint_plan_toeplitz(nlint_plan p, void *stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (p->algorithm == 2)
        return fail(NLINT_EUNSUPPORTED, "nlint_plan_toeplitz: not for an Algorithm 2 plan");
    if (p->toeplitz) return NLINT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int d = p->d, n = p->n_fine;
    const int64_t N = p->N, nh = n / 2 + 1;
    const size_t es = p->prec == NLINT_FP32 ? 4 : 8, cs = 2 * es;
    const int64_t half_cells = (d == 3) ? nh * n * n : nh * n;
    const int64_t full_cells = (d == 3) ? (int64_t)n * n * n : (int64_t)n * n;
    const int64_t grid = (d == 3) ? N * N * N : N * N;
    // ones (the convolution needs no deconvolution), the kernel's real half grid
    if ((rc = upload_ones(p))) return rc;
    CK(cudaMalloc(&p->d_khat, (size_t)half_cells * es));
    struct Tmp {
        void *kbuf = nullptr, *c = nullptr, *u = nullptr;
        ~Tmp() {
            if (kbuf) cudaFree(kbuf);
            if (c) cudaFree(c);
            if (u) cudaFree(u);
        }
    } t;
    CK(cudaMalloc(&t.kbuf, (size_t)half_cells * cs));
    CK(cudaMalloc(&t.c, (size_t)p->Nf * cs));
    CK(cudaMalloc(&t.u, (size_t)grid * es));
    CK(cudaMemsetAsync(t.kbuf, 0, (size_t)full_cells * es, s));

    // K(dx) = h^d Re sum_j W_j exp(i k_j . dx) for dx in [-N, N)^d cells, assembled from 2^d
    // type-1 evaluations of W_j exp(i k_j . delta) (delta = +-N/2 cells per axis) on the grid
    const double hd = std::pow(p->h, d);
    std::vector<double> ch(2 * (size_t)p->Nf);
    std::vector<float> cf;
    for (int sh = 0; sh < (1 << d); sh++) {
        int sgn[3] = {0, 0, 0};  // per node component (x, y, z)
        for (int c = 0; c < d; c++) sgn[c] = (sh >> c) & 1 ? 1 : -1;
        for (int64_t j = 0; j < p->Nf; j++) {
            double ph = 0.0;
            for (int c = 0; c < d; c++) ph += p->k_canon[(size_t)j * d + c] * sgn[c] * 0.5 * (double)N * p->h;
            ch[2 * j] = p->W_canon[j] * std::cos(ph);
            ch[2 * j + 1] = p->W_canon[j] * std::sin(ph);
        }
        if (p->prec == NLINT_FP32) {
            cf.assign(ch.begin(), ch.end());
            CK(cudaMemcpyAsync(t.c, cf.data(), cf.size() * 4, cudaMemcpyHostToDevice, s));
        } else {
            CK(cudaMemcpyAsync(t.c, ch.data(), ch.size() * 8, cudaMemcpyHostToDevice, s));
        }
        rc = nlint_type1(p, t.c, t.u, s);
        if (rc) return rc;
        // block cell i (centred index m = i - N/2) holds dx = m + sgn N/2; centred n-array index
        // dx + n/2; array axis a pairs with node component d - 1 - a
        int offs[3] = {0, 0, 0};
        for (int a = 0; a < d; a++) offs[a] = (int)(n / 2 - N / 2 + sgn[d - 1 - a] * (N / 2));
        const int3 off = (d == 3) ? make_int3(offs[0], offs[1], offs[2]) : make_int3(offs[0], 0, offs[1]);
        if (p->prec == NLINT_FP32) CK(launch_place_block<float>(d, N, n, off, t.u, hd, t.kbuf, s));
        else CK(launch_place_block<double>(d, N, n, off, t.u, hd, t.kbuf, s));
        CK(cudaStreamSynchronize(s));  // the host buffer is rewritten for the next shift
    }

    // K_hat = DFT of the circular kernel (forward passes, all n entries, no deconvolution)
    auto kpass = [&](PassDesc &pd, int in_kind, int out_kind) {
        std::memset(&pd, 0, sizeof(pd));
        pd.n = n;
        make_radix(n, pd);
        pd.sign = -1;
        pd.N = n;
        pd.dim = d;
        pd.fac = p->d_fac1;
        pd.in_kind = in_kind;
        pd.out_kind = out_kind;
    };
    PassDesc K1, K2, K3;
    kpass(K1, IN_REAL_MODES, OUT_CPLX_HALF);
    kpass(K3, IN_CPLX_MODES, OUT_CPLX_FULL);
    const void *kout;
    if (d == 3) {
        K1.I = (int64_t)n * n; K1.n_outer = 1; K1.in_sa = (int64_t)n * n; K1.out_sa = (int64_t)n * n;
        kpass(K2, IN_CPLX_MODES, OUT_CPLX_FULL);
        K2.I = n; K2.n_outer = nh; K2.in_so = (int64_t)n * n; K2.in_sa = n; K2.out_so = (int64_t)n * n; K2.out_sa = n;
        K3.I = nh * n; K3.in_so = n; K3.out_so = n;
        config_pass(K1, p->prec, false, p->fft_sched);
        config_pass(K2, p->prec, false, p->fft_sched);
        config_pass(K3, p->prec, true, p->fft_sched);
        if (p->prec == NLINT_FP32) {
            CK(launch_colpass<float>(K1, t.kbuf, p->d_bufG, p->d_tw, s));
            CK(launch_colpass<float>(K2, p->d_bufG, t.kbuf, p->d_tw, s));
            CK(launch_rowpass<float>(K3, t.kbuf, p->d_bufG, p->d_tw, s));
        } else {
            CK(launch_colpass<double>(K1, t.kbuf, p->d_bufG, p->d_tw, s));
            CK(launch_colpass<double>(K2, p->d_bufG, t.kbuf, p->d_tw, s));
            CK(launch_rowpass<double>(K3, t.kbuf, p->d_bufG, p->d_tw, s));
        }
        kout = p->d_bufG;
    } else {
        K1.I = n; K1.n_outer = 1; K1.in_sa = n; K1.out_sa = n;
        K3.I = nh; K3.in_so = n; K3.out_so = n;
        config_pass(K1, p->prec, false, p->fft_sched);
        config_pass(K3, p->prec, true, p->fft_sched);
        if (p->prec == NLINT_FP32) {
            CK(launch_colpass<float>(K1, t.kbuf, p->d_bufG, p->d_tw, s));
            CK(launch_rowpass<float>(K3, p->d_bufG, t.kbuf, p->d_tw, s));
        } else {
            CK(launch_colpass<double>(K1, t.kbuf, p->d_bufG, p->d_tw, s));
            CK(launch_rowpass<double>(K3, p->d_bufG, t.kbuf, p->d_tw, s));
        }
        kout = t.kbuf;
    }
    // the inverse passes are unnormalised: fold 1/n^d into K_hat
    const double inv = 1.0 / (double)full_cells;
    if (p->prec == NLINT_FP32) CK(launch_extract_real<float>(half_cells, kout, inv, p->d_khat, s));
    else CK(launch_extract_real<double>(half_cells, kout, inv, p->d_khat, s));
    CK(cudaStreamSynchronize(s));

    conv_passes(p);
    p->ws_bytes += (size_t)half_cells * es + (size_t)std::max<int64_t>(N, n) * es;
    p->toeplitz = true;
    return NLINT_OK;
}

int nlint_eval_toeplitz(nlint_plan p, const void *rho, void *u, double lambda, double *E_dev,
                        void *stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!rho || !u) return fail(NLINT_EINVAL, "NULL rho or u");
    if (p->algorithm == 2)
        return fail(NLINT_EUNSUPPORTED, "nlint_eval_toeplitz: not for an Algorithm 2 plan");
    if (!p->toeplitz) return fail(NLINT_EINVAL, "nlint_plan_toeplitz has not been called on this plan");
    cudaStream_t s = (cudaStream_t)stream;
    return p->prec == NLINT_FP32 ? run_toeplitz<float>(p, rho, u, lambda, E_dev, s)
                                 : run_toeplitz<double>(p, rho, u, lambda, E_dev, s);
}

int nlint_energy_only(nlint_plan p, const void *rho, double lambda, double *E_dev, double *E_host,
                      void *stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!rho) return fail(NLINT_EINVAL, "NULL rho");
    if (p->algorithm == 2)
        return fail(NLINT_EUNSUPPORTED, "nlint_energy_only: not for an Algorithm 2 plan");
    cudaStream_t s = (cudaStream_t)stream;
    p->ev_used = 0;
    // E = (lambda/2) sum_j W_j |rho_hat_j|^2 over the full node set = lambda sum over the half
    // set (W and |rho_hat| are even under k -> -k); the kernel sums (h^d W_j) |rho_hat_j/h^d|^2
    const double scale = lambda * std::pow(p->h, p->d);
    if (p->prec == NLINT_FP32) {
        if ((rc = run_type2<float>(p, rho, s))) return rc;
        CK(launch_interp<float>(node_desc(p), p->d_bufG, nullptr, 1, s, p->d_epart));
    } else {
        if ((rc = run_type2<double>(p, rho, s))) return rc;
        CK(launch_interp<double>(node_desc(p), p->d_bufG, nullptr, 1, s, p->d_epart));
    }
    double *E = E_dev ? E_dev : p->d_E;
    const int nparts = (int)(p->ngsub ? p->ngsub : p->nsub);  // one partial per interpolation CTA
    CK(launch_energy_final(p->d_epart, nparts, scale, E, s));
    p->launches += 1 + energy_final_kernels(nparts);
    if (E_host) {
        CK(cudaMemcpyAsync(E_host, E, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return NLINT_OK;
}

int nlint_eval_host(nlint_plan p, const void *rho_host, void *u_host, double lambda,
                    double *E_host, void *stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!rho_host || !u_host) return fail(NLINT_EINVAL, "NULL rho or u");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t count = 1;
    for (int a = 0; a < p->d; a++) count *= p->N;
    const size_t bytes = (size_t)count * (p->prec == NLINT_FP32 ? 4 : 8);
    if (!p->d_rho_io) CK(cudaMalloc(&p->d_rho_io, bytes));
    if (!p->d_u_io) CK(cudaMalloc(&p->d_u_io, bytes));
    CK(cudaMemcpyAsync(p->d_rho_io, rho_host, bytes, cudaMemcpyHostToDevice, s));
    rc = p->prec == NLINT_FP32 ? run_eval<float>(p, p->d_rho_io, p->d_u_io, lambda, p->d_E, s)
                               : run_eval<double>(p, p->d_rho_io, p->d_u_io, lambda, p->d_E, s);
    if (rc) return rc;
    CK(cudaMemcpyAsync(u_host, p->d_u_io, bytes, cudaMemcpyDeviceToHost, s));
    if (E_host) CK(cudaMemcpyAsync(E_host, p->d_E, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return NLINT_OK;
}

int nlint_eval_host_many(nlint_plan p, int count, const void *const *rho_host, void *const *u_host,
                         double lambda, double *E_host, void *stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (count <= 0 || !rho_host || !u_host)
        return fail(NLINT_EINVAL, "count must be positive and rho_host, u_host non-NULL");
    for (int k = 0; k < count; k++)
        if (!rho_host[k] || !u_host[k]) return fail(NLINT_EINVAL, "NULL rho_host[k] or u_host[k]");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t cells = 1;
    for (int a = 0; a < p->d; a++) cells *= p->N;
    const size_t bytes = (size_t)cells * (p->prec == NLINT_FP32 ? 4 : 8);
    if (!p->s_in) {
        CK(cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking));
        for (cudaEvent_t &e : p->ev_io) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    for (int b = 0; b < 2; b++) {
        if (!p->d_rho_st[b]) CK(cudaMalloc(&p->d_rho_st[b], bytes));
        if (!p->d_u_st[b]) CK(cudaMalloc(&p->d_u_st[b], bytes));
    }
    if (E_host && p->nEm < count) {
        if (p->d_Em) CK(cudaFree(p->d_Em));
        p->d_Em = nullptr;
        p->nEm = 0;
        CK(cudaMalloc((void **)&p->d_Em, sizeof(double) * (size_t)count));
        p->nEm = count;
    }
    cudaEvent_t *ev_in = p->ev_io, *ev_comp = p->ev_io + 2, *ev_out = p->ev_io + 4, ev_fj = p->ev_io[6];
    CK(cudaEventRecord(ev_fj, s));  // the copies follow the work already queued on `stream`
    CK(cudaStreamWaitEvent(p->s_in, ev_fj, 0));
    CK(cudaStreamWaitEvent(p->s_out, ev_fj, 0));
    for (int k = 0; k < count; k++) {
        const int b = k & 1;
        // density k into staging buffer b, once evaluation k-2 (the last reader of b) is done
        CK(cudaStreamWaitEvent(p->s_in, ev_comp[b], 0));
        CK(cudaMemcpyAsync(p->d_rho_st[b], rho_host[k], bytes, cudaMemcpyHostToDevice, p->s_in));
        CK(cudaEventRecord(ev_in[b], p->s_in));
        // evaluation k, once its density has arrived and u_{k-2} has left staging buffer b
        CK(cudaStreamWaitEvent(s, ev_in[b], 0));
        CK(cudaStreamWaitEvent(s, ev_out[b], 0));
        double *E = E_host ? p->d_Em + k : nullptr;
        rc = p->prec == NLINT_FP32 ? run_eval<float>(p, p->d_rho_st[b], p->d_u_st[b], lambda, E, s)
                                   : run_eval<double>(p, p->d_rho_st[b], p->d_u_st[b], lambda, E, s);
        if (rc) return rc;
        CK(cudaEventRecord(ev_comp[b], s));
        // u_k back to the host while evaluation k+1 runs
        CK(cudaStreamWaitEvent(p->s_out, ev_comp[b], 0));
        CK(cudaMemcpyAsync(u_host[k], p->d_u_st[b], bytes, cudaMemcpyDeviceToHost, p->s_out));
        CK(cudaEventRecord(ev_out[b], p->s_out));
    }
    CK(cudaEventRecord(ev_fj, p->s_out));  // join both copy streams back into `stream`
    CK(cudaStreamWaitEvent(s, ev_fj, 0));
    CK(cudaEventRecord(ev_fj, p->s_in));
    CK(cudaStreamWaitEvent(s, ev_fj, 0));
    if (E_host) CK(cudaMemcpyAsync(E_host, p->d_Em, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return NLINT_OK;
}

int nlint_type2(nlint_plan p, const void *rho, void *rho_hat, void *stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!rho || !rho_hat) return fail(NLINT_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    p->ev_used = 0;
    const double hd = std::pow(p->h, p->d);
    if (p->prec == NLINT_FP32) {
        if ((rc = run_type2<float>(p, rho, s))) return rc;
        CK(launch_interp<float>(node_desc(p), p->d_bufG, p->d_c, 0, s));
        CK(launch_scatter_canonical<float>(p->Mh, p->d_c, p->d_perm, p->d_mirror, hd, rho_hat, s));
        p->launches += 2;
    } else {
        if ((rc = run_type2<double>(p, rho, s))) return rc;
        CK(launch_interp<double>(node_desc(p), p->d_bufG, p->d_c, 0, s));
        CK(launch_scatter_canonical<double>(p->Mh, p->d_c, p->d_perm, p->d_mirror, hd, rho_hat, s));
        p->launches += 2;
    }
    return NLINT_OK;
}

int nlint_type1(nlint_plan p, const void *c, void *u, void *stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!c || !u) return fail(NLINT_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    p->ev_used = 0;
    p->launches += 1;
    if (p->d_bufH && (rc = clear_spread_grid(p, s))) return rc;
    if (p->prec == NLINT_FP32) {
        CK(launch_gather_canonical<float>(p->Mh, c, p->d_perm, p->d_mirror, p->d_c, s));
        return run_type1<float>(p, u, nullptr, s);
    }
    CK(launch_gather_canonical<double>(p->Mh, c, p->d_perm, p->d_mirror, p->d_c, s));
    return run_type1<double>(p, u, nullptr, s);
}

int nlint_set_stage_timing(nlint_plan p, int enable) {
    if (!p) return fail(NLINT_EINVAL, "plan is NULL");
    p->timing = enable != 0;
    return NLINT_OK;
}

int nlint_stage_times(nlint_plan p, float *ms, const char **names, int max_stages, int *n_stages) {
    if (!p) return fail(NLINT_EINVAL, "plan is NULL");
    const int k = std::max(0, p->ev_used - 1);
    if (n_stages) *n_stages = k;
    if (k == 0) return NLINT_OK;
    CK(cudaEventSynchronize(p->ev[p->ev_used - 1]));
    for (int i = 0; i < k && i < max_stages; i++) {
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, p->ev[i], p->ev[i + 1]));
        if (ms) ms[i] = t;
        if (names) names[i] = p->ev_names[i + 1];
    }
    return NLINT_OK;
}

int nlint_launch_count(nlint_plan p, int64_t *count) {
    if (!p || !count) return fail(NLINT_EINVAL, "NULL argument");
    *count = p->launches;
    return NLINT_OK;
}

const char *nlint_last_error(void) { return g_err.c_str(); }

}  // extern "C"
