// Node-order permutations and the energy reduction (step a8 of the path; Remark 3.3), and the
// dispatch of the interpolation / spreading launchers to their per-(precision, dimension)
// translation units (node_kernels.cuh).
#include "common.cuh"
#include "internal.h"

namespace nlint {

int tile_cells(const NodeDesc &nd) {
    return nd.d == 3 ? nd.T[0] * nd.T[1] * nd.T[2] : nd.T[0] * nd.T[1];
}

// Shared memory of the interpolation / spreading kernels: the tile (real and imaginary
// planes) plus, for FP64, one table of 2 x 3 x NODE_MAXW kernel values per warp (two nodes
// at a time).  FP32 kernels evaluate the stencil values in registers and exchange them by
// warp shuffles.
size_t node_smem_for(int prec, int d, int w, int bs) {
    const size_t s = prec == NLINT_FP32 ? 4 : 8;  // tile cell: float/int32 or double/int64
    // 3D: T0 x T1 rows of tile_pitch cells (the pitch pads FP32 rows against bank conflicts)
    size_t cells = 1;
    for (int a = 0; a < d - 1; a++) cells *= (size_t)(bin_dim(d, bs, a) + w - 1);
    cells *= (size_t)tile_pitch(prec == NLINT_FP64, d, w, bs);
    const size_t table = prec == NLINT_FP32 ? 0 : (size_t)(NODE_THREADS / 32) * 6 * NODE_MAXW * s;
    return 2 * cells * s + table;
}

size_t node_smem(const NodeDesc &nd, int prec) {
    return node_smem_for(prec, nd.d, nd.w, nd.bin_shape);
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
__global__ void __launch_bounds__(256) energy_partials_kernel(int64_t count, const T *__restrict__ u,
                                                              const T *__restrict__ rho,
                                                              double2 *__restrict__ partials) {
    __shared__ double sh[2 * 32];
    EAcc<T> acc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        acc.add(u[i], rho[i]);
    const double2 tot = energy_block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// One CTA of 1024 threads folds the partials: thread t takes partials t, t+1024, ... in
// order, then a fixed shuffle tree combines the threads.  The result does not depend on
// timing, so repeated evaluations give identical energies.
// Energy fold in two stages, so the FP64 compensated arithmetic (a small fraction of the FP32
// rate on this GPU) is spread over many SMs: warp b folds partials [b per, (b + 1) per) into
// out[b], then one CTA folds those.  The order is fixed by the indices (deterministic).
__global__ void __launch_bounds__(32) energy_fold_kernel(const double2 *__restrict__ partials,
                                                         int nparts, int per,
                                                         double2 *__restrict__ out) {
    pdl_wait();  // (launched by launch_pdl)
    pdl_trigger();
    KSum acc;
    acc.init();
    const int a = blockIdx.x * per, e = min(a + per, nparts);
    for (int q = a + (int)threadIdx.x; q < e; q += 32) acc.merge(partials[q].x, partials[q].y);
    ksum_warp(acc);
    if (threadIdx.x == 0) out[blockIdx.x] = make_double2(acc.s, acc.c);
}

__global__ void __launch_bounds__(1024) energy_final_kernel(const double2 *__restrict__ partials,
                                                            int nparts, double scale,
                                                            double *__restrict__ E) {
    pdl_wait();  // (launched by launch_pdl)
    pdl_trigger();
    __shared__ double sh[2 * 32];
    KSum acc;
    acc.init();
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) acc.merge(partials[q].x, partials[q].y);
    KSum tot = ksum_block(acc, sh);
    if (threadIdx.x == 0) *E = scale * tot.value();
}

// Toeplitz kernel assembly: K[a] = scale * u[i] for an N^d block u placed in an n^d array at
// cell offsets off = (slowest axis, middle axis, fastest axis); in 2D off.y is unused.
template <typename T>
__global__ void place_block_kernel(int d, int64_t N, int64_t n, int3 off, const T *__restrict__ u,
                                   double scale, T *__restrict__ K) {
    const int64_t cnt = (d == 3) ? N * N * N : N * N;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int64_t ix = i % N, r = i / N;
    int64_t a;
    if (d == 3) {
        const int64_t iy = r % N, iz = r / N;
        a = ((iz + off.x) * n + (iy + off.y)) * n + (ix + off.z);
    } else {
        a = (r + off.x) * n + (ix + off.z);
    }
    K[a] = (T)(scale * (double)u[i]);
}

// khat[i] = scale * Re(G[i])
template <typename T>
__global__ void extract_real_kernel(int64_t cnt, const cx_t<T> *__restrict__ G, double scale,
                                    T *__restrict__ khat) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) khat[i] = (T)(scale * (double)G[i].x);
}

// --------------------------------------------------------------------------- launchers
template <typename T>
cudaError_t launch_place_block(int d, int64_t N, int64_t n, int3 off, const void *u, double scale,
                               void *K, cudaStream_t s) {
    const int64_t cnt = (d == 3) ? N * N * N : N * N;
    place_block_kernel<T><<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(d, N, n, off, (const T *)u,
                                                                       scale, (T *)K);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extract_real(int64_t cnt, const void *G, double scale, void *khat, cudaStream_t s) {
    extract_real_kernel<T><<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(cnt, (const cx_t<T> *)G, scale,
                                                                         (T *)khat);
    return cudaGetLastError();
}

static inline unsigned nblk(int64_t M, int t) { return (unsigned)((M + t - 1) / t); }

// Dispatch on the plan's dimension and bin shape to the compiled combinations
// (bin_shape_built): FP32 3D shapes 1, 3, 4; FP64 3D shapes 1, 2; 2D shape 1.
template <typename T>
cudaError_t launch_interp(const NodeDesc &nd, const void *G, void *c_out, int apply_W,
                          cudaStream_t s, double2 *epart) {
    constexpr bool F64 = sizeof(T) == 8;
    if (nd.d == 2) return nd.bin_shape == 1 ? launch_interp_bs<T, 2, 1>(nd, G, c_out, apply_W, epart, s)
                                            : cudaErrorInvalidValue;
    switch (nd.bin_shape) {
        case 1: return launch_interp_bs<T, 3, 1>(nd, G, c_out, apply_W, epart, s);
        case 2: if constexpr (F64) return launch_interp_bs<T, 3, 2>(nd, G, c_out, apply_W, epart, s);
                break;
        case 3: if constexpr (!F64) return launch_interp_bs<T, 3, 3>(nd, G, c_out, apply_W, epart, s);
                break;
        case 4: if constexpr (!F64) return launch_interp_bs<T, 3, 4>(nd, G, c_out, apply_W, epart, s);
                break;
        default: break;
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_spread(const NodeDesc &nd, const void *c_in, void *Hext, cudaStream_t s) {
    constexpr bool F64 = sizeof(T) == 8;
    if (nd.d == 2) return nd.bin_shape == 1 ? launch_spread_bs<T, 2, 1>(nd, c_in, Hext, s)
                                            : cudaErrorInvalidValue;
    switch (nd.bin_shape) {
        case 1: return launch_spread_bs<T, 3, 1>(nd, c_in, Hext, s);
        case 2: if constexpr (F64) return launch_spread_bs<T, 3, 2>(nd, c_in, Hext, s);
                break;
        case 3: if constexpr (!F64) return launch_spread_bs<T, 3, 3>(nd, c_in, Hext, s);
                break;
        case 4: if constexpr (!F64) return launch_spread_bs<T, 3, 4>(nd, c_in, Hext, s);
                break;
        default: break;
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_crowd_merge(const NodeDesc &nd, void *Hext, cudaStream_t s) {
    return nd.d == 3 ? launch_crowd_merge_d<T, 3>(nd, Hext, s) : launch_crowd_merge_d<T, 2>(nd, Hext, s);
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

static constexpr int FOLD_DIRECT = 128, FOLD_WARPS = 64;

int energy_final_kernels(int nparts) { return nparts <= FOLD_DIRECT ? 1 : 2; }

cudaError_t launch_energy_final(const double2 *partials, int nparts, double scale, double *E,
                                cudaStream_t s) {
    if (nparts <= FOLD_DIRECT) {
        const cudaError_t e = launch_pdl(energy_final_kernel, dim3(1), dim3(FOLD_DIRECT), 0, s, partials,
                                         nparts, scale, E);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    const int per = (nparts + FOLD_WARPS - 1) / FOLD_WARPS;
    const int g = (nparts + per - 1) / per;  // <= FOLD_WARPS
    double2 *mid = const_cast<double2 *>(partials) + nparts;
    cudaError_t e = launch_pdl(energy_fold_kernel, dim3(g), dim3(32), 0, s, partials, nparts, per, mid);
    if (e != cudaSuccess) return e;
    e = launch_pdl(energy_final_kernel, dim3(1), dim3(FOLD_WARPS), 0, s, (const double2 *)mid, g, scale, E);
    return e != cudaSuccess ? e : cudaGetLastError();
}

#define NLINT_INST(T)                                                                              \
    template cudaError_t launch_interp<T>(const NodeDesc &, const void *, void *, int, cudaStream_t, \
                                          double2 *);                                             \
    template cudaError_t launch_spread<T>(const NodeDesc &, const void *, void *, cudaStream_t);      \
    template cudaError_t launch_crowd_merge<T>(const NodeDesc &, void *, cudaStream_t);              \
    template cudaError_t launch_place_block<T>(int, int64_t, int64_t, int3, const void *, double,    \
                                               void *, cudaStream_t);                                \
    template cudaError_t launch_extract_real<T>(int64_t, const void *, double, void *, cudaStream_t); \
    template cudaError_t launch_scatter_canonical<T>(int64_t, const void *, const int32_t *,         \
                                                     const int32_t *, double, void *, cudaStream_t); \
    template cudaError_t launch_gather_canonical<T>(int64_t, const void *, const int32_t *,          \
                                                    const int32_t *, void *, cudaStream_t);          \
    template cudaError_t launch_energy_partials<T>(int64_t, const void *, const void *, double2 *,   \
                                                   int, cudaStream_t);
NLINT_INST(float)
NLINT_INST(double)

}  // namespace nlint
