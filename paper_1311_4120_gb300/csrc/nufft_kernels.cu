// Type-2 interpolation, multiply, type-1 spreading and the energy reduction (steps a3, a4,
// a5 and a8 of the path; Algorithm 1, eq. 3.2 and eq. 3.7, Remark 3.3).
//
// Spreading kernel: the "exponential of semicircle" function of Barnett, Magland and
// af Klinteberg (SIAM J. Sci. Comput. 2019), phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on
// |z| <= 1, with z = (l - g) / (w/2) for fine cell l and node position g (fine-cell units).
//
// Only the half node set S+ (k on the positive side of the slowest array axis) is
// processed: rho_hat(-k) = conj(rho_hat(k)) for a real density, and the mirrored nodes'
// spreading is restored by the fold in the first inverse FFT pass.  The fine grid G holds
// the planes lz = 0..n/2 of the slowest axis; a stencil cell outside that range is read as
// conj(G[-l]).  The spread grid H+ is stored on planes lz = -pad..n/2+pad.
#include "common.cuh"
#include "internal.h"

namespace nlint {

static constexpr int MAXW = 16;

template <typename T>
__device__ __forceinline__ T es_kernel(T z, T beta) {
    const T s = T(1) - z * z;
    return s > T(0) ? exp(beta * (sqrt(s) - T(1))) : T(0);
}

__device__ __forceinline__ int wrapn(int l, int n) {
    int r = l % n;
    return r < 0 ? r + n : r;
}

template <typename T, int D>
__device__ __forceinline__ void node_weights(const NodeDesc &nd, int64_t j, T (&ker)[D][MAXW],
                                             int (&l0)[D]) {
    const T *frac = reinterpret_cast<const T *>(nd.frac);
    const T half = T(nd.w) * T(0.5);
    const T beta = T(nd.beta);
#pragma unroll
    for (int a = 0; a < D; a++) {
        const T fr = frac[a * nd.M + j];
        l0[a] = nd.l0[a * nd.M + j];
#pragma unroll
        for (int q = 0; q < MAXW; q++) {
            if (q < nd.w) ker[a][q] = es_kernel<T>((T(q) - fr) / half, beta);
        }
    }
}

// Read G at (lz, ly, lx) of the full periodic grid from its stored half (planes 0..n/2).
template <typename T, int D>
__device__ __forceinline__ cx_t<T> fetch_half(const cx_t<T> *__restrict__ G, int n, int lz, int ly,
                                              int lx) {
    if (lz >= 0 && lz <= n / 2) {
        if (D == 3) return G[((int64_t)lz * n + wrapn(ly, n)) * n + wrapn(lx, n)];
        return G[(int64_t)lz * n + wrapn(lx, n)];
    }
    const int mz = lz < 0 ? -lz : n - lz;
    if (D == 3) return cconj(G[((int64_t)mz * n + wrapn(-ly, n)) * n + wrapn(-lx, n)]);
    return cconj(G[(int64_t)mz * n + wrapn(-lx, n)]);
}

template <typename T, int D>
__global__ void __launch_bounds__(128) interp_kernel(NodeDesc nd, const cx_t<T> *__restrict__ G,
                                                     cx_t<T> *__restrict__ c_out, int apply_W) {
    using T2 = cx_t<T>;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nd.M) return;
    T ker[D][MAXW];
    int l0[D];
    node_weights<T, D>(nd, j, ker, l0);
    const int w = nd.w, n = nd.n;
    T2 acc = czero<T2>();
    if (D == 3) {
        for (int qa = 0; qa < w; qa++) {
            for (int qb = 0; qb < w; qb++) {
                const T wab = ker[0][qa] * ker[1 % D][qb];
                for (int qc = 0; qc < w; qc++) {
                    const T2 g = fetch_half<T, D>(G, n, l0[0] + qa, l0[1 % D] + qb, l0[2 % D] + qc);
                    const T wt = wab * ker[2 % D][qc];
                    acc.x += wt * g.x;
                    acc.y += wt * g.y;
                }
            }
        }
    } else {
        for (int qa = 0; qa < w; qa++) {
            for (int qc = 0; qc < w; qc++) {
                const T2 g = fetch_half<T, D>(G, n, l0[0] + qa, 0, l0[1 % D] + qc);
                const T wt = ker[0][qa] * ker[1 % D][qc];
                acc.x += wt * g.x;
                acc.y += wt * g.y;
            }
        }
    }
    if (apply_W) acc = cscale(acc, reinterpret_cast<const T *>(nd.W)[j]);
    c_out[j] = acc;
}

template <typename T, int D>
__global__ void __launch_bounds__(128) spread_kernel(NodeDesc nd, const cx_t<T> *__restrict__ c_in,
                                                     cx_t<T> *__restrict__ H) {
    using T2 = cx_t<T>;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nd.M) return;
    T ker[D][MAXW];
    int l0[D];
    node_weights<T, D>(nd, j, ker, l0);
    const int w = nd.w, n = nd.n, pad = nd.pad;
    const T2 c = c_in[j];
    T *Hr = reinterpret_cast<T *>(H);
    for (int qa = 0; qa < w; qa++) {
        const int64_t plane = (int64_t)(l0[0] + qa + pad);
        if (D == 3) {
            for (int qb = 0; qb < w; qb++) {
                const T wab = ker[0][qa] * ker[1 % D][qb];
                const int64_t rowb = (plane * n + wrapn(l0[1 % D] + qb, n)) * n;
                for (int qc = 0; qc < w; qc++) {
                    const T wt = wab * ker[2 % D][qc];
                    const int64_t idx = rowb + wrapn(l0[2 % D] + qc, n);
                    atomicAdd(Hr + 2 * idx, wt * c.x);
                    atomicAdd(Hr + 2 * idx + 1, wt * c.y);
                }
            }
        } else {
            for (int qc = 0; qc < w; qc++) {
                const T wt = ker[0][qa] * ker[1 % D][qc];
                const int64_t idx = plane * n + wrapn(l0[1 % D] + qc, n);
                atomicAdd(Hr + 2 * idx, wt * c.x);
                atomicAdd(Hr + 2 * idx + 1, wt * c.y);
            }
        }
    }
}

// out[perm[j]] = scale * v_j, out[mirror[j]] = scale * conj(v_j)
template <typename T>
__global__ void scatter_canonical_kernel(int64_t M, const cx_t<T> *__restrict__ v,
                                         const int32_t *__restrict__ perm,
                                         const int32_t *__restrict__ mirror, T scale,
                                         cx_t<T> *__restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const cx_t<T> x = cscale(v[j], scale);
    out[perm[j]] = x;
    out[mirror[j]] = cconj(x);
}

// c_half[j] = (c[perm[j]] + conj(c[mirror[j]])) / 2
template <typename T>
__global__ void gather_canonical_kernel(int64_t M, const cx_t<T> *__restrict__ c,
                                        const int32_t *__restrict__ perm,
                                        const int32_t *__restrict__ mirror,
                                        cx_t<T> *__restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    out[j] = cscale(cadd(c[perm[j]], cconj(c[mirror[j]])), T(0.5));
}

template <typename T>
__global__ void energy_partials_kernel(int64_t count, const T *__restrict__ u,
                                       const T *__restrict__ rho, double2 *__restrict__ partials) {
    __shared__ double sh[2 * 256];
    KSum acc;
    acc.init();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        acc.add((double)u[i] * (double)rho[i]);
    sh[2 * threadIdx.x] = acc.s;
    sh[2 * threadIdx.x + 1] = acc.c;
    __syncthreads();
    if (threadIdx.x == 0) {
        KSum tot;
        tot.init();
        for (int q = 0; q < (int)blockDim.x; q++) {
            tot.add(sh[2 * q]);
            tot.add(sh[2 * q + 1]);
        }
        partials[blockIdx.x] = make_double2(tot.s, tot.c);
    }
}

// One thread sums the partials in index order: the result does not depend on timing.
__global__ void energy_final_kernel(const double2 *__restrict__ partials, int nparts,
                                    double scale, double *__restrict__ E) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    KSum tot;
    tot.init();
    for (int q = 0; q < nparts; q++) {
        tot.add(partials[q].x);
        tot.add(partials[q].y);
    }
    *E = scale * tot.value();
}

// --------------------------------------------------------------------------- launchers
static inline unsigned nblk(int64_t M, int t) { return (unsigned)((M + t - 1) / t); }

template <typename T>
cudaError_t launch_interp(const NodeDesc &nd, const void *G, void *c_out, int apply_W,
                          cudaStream_t s) {
    if (nd.M == 0) return cudaSuccess;
    if (nd.d == 3)
        interp_kernel<T, 3><<<nblk(nd.M, 128), 128, 0, s>>>(nd, (const cx_t<T> *)G, (cx_t<T> *)c_out, apply_W);
    else
        interp_kernel<T, 2><<<nblk(nd.M, 128), 128, 0, s>>>(nd, (const cx_t<T> *)G, (cx_t<T> *)c_out, apply_W);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spread(const NodeDesc &nd, const void *c_in, void *Hext, cudaStream_t s) {
    if (nd.M == 0) return cudaSuccess;
    if (nd.d == 3)
        spread_kernel<T, 3><<<nblk(nd.M, 128), 128, 0, s>>>(nd, (const cx_t<T> *)c_in, (cx_t<T> *)Hext);
    else
        spread_kernel<T, 2><<<nblk(nd.M, 128), 128, 0, s>>>(nd, (const cx_t<T> *)c_in, (cx_t<T> *)Hext);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter_canonical(int64_t M, const void *vals, const int32_t *perm,
                                     const int32_t *mirror, double scale, void *out,
                                     cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    scatter_canonical_kernel<T><<<nblk(M, 256), 256, 0, s>>>(M, (const cx_t<T> *)vals, perm, mirror,
                                                            (T)scale, (cx_t<T> *)out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_canonical(int64_t M, const void *c_canon, const int32_t *perm,
                                    const int32_t *mirror, void *c_half, cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    gather_canonical_kernel<T><<<nblk(M, 256), 256, 0, s>>>(M, (const cx_t<T> *)c_canon, perm, mirror,
                                                           (cx_t<T> *)c_half);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_energy_partials(int64_t count, const void *u, const void *rho,
                                   double2 *partials, int nblocks, cudaStream_t s) {
    energy_partials_kernel<T><<<nblocks, 256, 0, s>>>(count, (const T *)u, (const T *)rho, partials);
    return cudaGetLastError();
}

cudaError_t launch_energy_final(const double2 *partials, int nparts, double scale, double *E,
                                cudaStream_t s) {
    energy_final_kernel<<<1, 32, 0, s>>>(partials, nparts, scale, E);
    return cudaGetLastError();
}

#define NLINT_INST(T)                                                                              \
    template cudaError_t launch_interp<T>(const NodeDesc &, const void *, void *, int, cudaStream_t); \
    template cudaError_t launch_spread<T>(const NodeDesc &, const void *, void *, cudaStream_t);      \
    template cudaError_t launch_scatter_canonical<T>(int64_t, const void *, const int32_t *,         \
                                                     const int32_t *, double, void *, cudaStream_t); \
    template cudaError_t launch_gather_canonical<T>(int64_t, const void *, const int32_t *,          \
                                                    const int32_t *, void *, cudaStream_t);          \
    template cudaError_t launch_energy_partials<T>(int64_t, const void *, const void *, double2 *,   \
                                                   int, cudaStream_t);
NLINT_INST(float)
NLINT_INST(double)

}  // namespace nlint
