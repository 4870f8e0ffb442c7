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

// Read G at (l0, l1[, l2]) of the full periodic fine grid from its stored half (planes
// 0..n/2 of axis 0), using G[-l] = conj(G[l]) for the other half.
template <typename T, int D>
__device__ __forceinline__ cx_t<T> fetch_half(const cx_t<T> *__restrict__ G, int n, int l0, int l1,
                                              int l2) {
    const int z = wrapn(l0, n);
    if (z <= n / 2) {
        if (D == 3) return G[((int64_t)z * n + wrapn(l1, n)) * n + wrapn(l2, n)];
        return G[(int64_t)z * n + wrapn(l1, n)];
    }
    const int mz = n - z;
    if (D == 3) return cconj(G[((int64_t)mz * n + wrapn(-l1, n)) * n + wrapn(-l2, n)]);
    return cconj(G[(int64_t)mz * n + wrapn(-l1, n)]);
}

int tile_cells(const NodeDesc &nd) {
    return nd.d == 3 ? nd.T[0] * nd.T[1] * nd.T[2] : nd.T[0] * nd.T[1];
}

static constexpr int SUB_THREADS = 256;

// Shared memory of the interpolation / spreading kernels: the tile (real and imaginary
// planes) plus one table of D x MAXW kernel values per warp.
size_t node_smem(const NodeDesc &nd, int prec) {
    const size_t s = prec == NLINT_FP32 ? 4 : 8;
    return 2 * (size_t)tile_cells(nd) * s + (size_t)(SUB_THREADS / 32) * 3 * MAXW * s;
}

// Kernel values of one node, computed by the lanes of the warp (D*w values, up to 48, so
// some lanes take two) into ker[a*MAXW+q] = phi((q - frac_a) / (w/2)) for stencil cell q on
// axis a.
template <typename T, int D>
__device__ __forceinline__ void warp_kernel_values(const NodeDesc &nd, int64_t j, int lane, T *ker) {
    const int w = nd.w;
    for (int t = lane; t < D * w; t += 32) {
        const int a = t / w, q = t - a * w;
        const T fr = reinterpret_cast<const T *>(nd.frac)[a * nd.M + j];
        ker[a * MAXW + q] = es_kernel<T>((T(q) - fr) / (T(w) * T(0.5)), T(nd.beta));
    }
}

// Type-2 interpolation (step a3) and the multiply by W_j (step a4): one CTA per subproblem
// stages its bin's tile of G in shared memory; each warp takes one node at a time, its lanes
// cover the stencil's (axis 1, axis 2) columns and run along axis 0, and a shuffle tree sums
// the lanes.  c_out is written in sorted (bin) order.
template <typename T, int D>
__global__ void __launch_bounds__(SUB_THREADS) interp_sub_kernel(NodeDesc nd,
                                                                const cx_t<T> *__restrict__ G,
                                                                cx_t<T> *__restrict__ c_out,
                                                                int apply_W) {
    using T2 = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ncell = (D == 3) ? nd.T[0] * nd.T[1] * nd.T[2] : nd.T[0] * nd.T[1];
    T *tr = reinterpret_cast<T *>(smem_raw);
    T *ti = tr + ncell;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T *ker = ti + ncell + wid * 3 * MAXW;
    const int4 sb = nd.subs[blockIdx.x];
    const int4 bo = nd.bins[sb.z];
    const int n = nd.n, w = nd.w;
    const int T1 = nd.T[1], T2n = (D == 3) ? nd.T[2] : 1;

    for (int cell = threadIdx.x; cell < ncell; cell += blockDim.x) {
        T2 v;
        if (D == 3) {
            const int a0 = cell / (T1 * T2n), rem = cell - a0 * T1 * T2n;
            const int a1 = rem / T2n, a2 = rem - a1 * T2n;
            v = fetch_half<T, 3>(G, n, bo.x + a0, bo.y + a1, bo.z + a2);
        } else {
            const int a0 = cell / T1, a1 = cell - a0 * T1;
            v = fetch_half<T, 2>(G, n, bo.x + a0, bo.y + a1, 0);
        }
        tr[cell] = v.x;
        ti[cell] = v.y;
    }
    __syncthreads();

    const int64_t M = nd.M;
    for (int i = wid; i < sb.y; i += nw) {
        const int64_t j = (int64_t)sb.x + i;
        warp_kernel_values<T, D>(nd, j, lane, ker);
        const int r0 = nd.l0[j] - bo.x, r1 = nd.l0[M + j] - bo.y;
        const int r2 = (D == 3) ? nd.l0[2 * M + j] - bo.z : 0;
        __syncwarp();
        T accr = T(0), acci = T(0);
        if (D == 3) {
            const int plane = T1 * T2n;
            for (int p = lane; p < w * w; p += 32) {
                const int q1 = p / w, q2 = p - q1 * w;
                int idx = (r0 * T1 + r1 + q1) * T2n + r2 + q2;
                T sr = T(0), si = T(0);
                for (int q0 = 0; q0 < w; q0++, idx += plane) {
                    const T k0 = ker[q0];
                    sr += k0 * tr[idx];
                    si += k0 * ti[idx];
                }
                const T k12 = ker[MAXW + q1] * ker[2 * MAXW + q2];
                accr += k12 * sr;
                acci += k12 * si;
            }
        } else {
            for (int p = lane; p < w * w; p += 32) {
                const int q0 = p / w, q1 = p - q0 * w;
                const int idx = (r0 + q0) * T1 + r1 + q1;
                const T k = ker[q0] * ker[MAXW + q1];
                accr += k * tr[idx];
                acci += k * ti[idx];
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            accr += __shfl_xor_sync(0xffffffffu, accr, off);
            acci += __shfl_xor_sync(0xffffffffu, acci, off);
        }
        if (lane == 0) {
            const T sc = apply_W ? reinterpret_cast<const T *>(nd.W)[j] : T(1);
            c_out[j] = cmake<T2>(accr * sc, acci * sc);
        }
        __syncwarp();
    }
}

__device__ __forceinline__ void atomic_add_cx(float2 *p, float re, float im) {
    atomicAdd(p, make_float2(re, im));
}
__device__ __forceinline__ void atomic_add_cx(double2 *p, double re, double im) {
    atomicAdd(&p->x, re);
    atomicAdd(&p->y, im);
}

// Type-1 spreading (step a5): one CTA per subproblem accumulates its nodes' stencils into a
// shared-memory tile with shared atomics (lanes of a warp cover distinct cells of one node),
// then adds the tile's nonzero cells to the extended spread grid with global atomics.  Tiles
// of crowded bins go to an FP64 accumulator instead (their cells receive up to 10^5 terms).
template <typename T, int D>
__global__ void __launch_bounds__(SUB_THREADS) spread_sub_kernel(NodeDesc nd,
                                                                const cx_t<T> *__restrict__ c_in,
                                                                cx_t<T> *__restrict__ H) {
    using T2 = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ncell = (D == 3) ? nd.T[0] * nd.T[1] * nd.T[2] : nd.T[0] * nd.T[1];
    T *tr = reinterpret_cast<T *>(smem_raw);
    T *ti = tr + ncell;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T *ker = ti + ncell + wid * 3 * MAXW;
    const int4 sb = nd.subs[blockIdx.x];
    const int4 bo = nd.bins[sb.z];
    const int n = nd.n, w = nd.w, pad = nd.pad;
    const int T1 = nd.T[1], T2n = (D == 3) ? nd.T[2] : 1;

    for (int cell = threadIdx.x; cell < ncell; cell += blockDim.x) {
        tr[cell] = T(0);
        ti[cell] = T(0);
    }
    __syncthreads();

    const int64_t M = nd.M;
    for (int i = wid; i < sb.y; i += nw) {
        const int64_t j = (int64_t)sb.x + i;
        warp_kernel_values<T, D>(nd, j, lane, ker);
        const int r0 = nd.l0[j] - bo.x, r1 = nd.l0[M + j] - bo.y;
        const int r2 = (D == 3) ? nd.l0[2 * M + j] - bo.z : 0;
        const T2 c = c_in[j];
        __syncwarp();
        if (D == 3) {
            const int plane = T1 * T2n;
            for (int p = lane; p < w * w; p += 32) {
                const int q1 = p / w, q2 = p - q1 * w;
                const T k12 = ker[MAXW + q1] * ker[2 * MAXW + q2];
                const T cr = c.x * k12, ci = c.y * k12;
                int idx = (r0 * T1 + r1 + q1) * T2n + r2 + q2;
                for (int q0 = 0; q0 < w; q0++, idx += plane) {
                    const T k0 = ker[q0];
                    atomicAdd(tr + idx, cr * k0);
                    atomicAdd(ti + idx, ci * k0);
                }
            }
        } else {
            for (int p = lane; p < w * w; p += 32) {
                const int q0 = p / w, q1 = p - q0 * w;
                const int idx = (r0 + q0) * T1 + r1 + q1;
                const T k = ker[q0] * ker[MAXW + q1];
                atomicAdd(tr + idx, c.x * k);
                atomicAdd(ti + idx, c.y * k);
            }
        }
        __syncwarp();
    }
    __syncthreads();

    const int slot = bo.w;
    const int nplanes = n / 2 + 1 + 2 * pad;
    for (int cell = threadIdx.x; cell < ncell; cell += blockDim.x) {
        const T vr = tr[cell], vi = ti[cell];
        if (vr == T(0) && vi == T(0)) continue;
        if (slot >= 0) {
            atomic_add_cx(nd.crowd + (int64_t)slot * ncell + cell, (double)vr, (double)vi);
            continue;
        }
        int64_t g;
        if (D == 3) {
            const int a0 = cell / (T1 * T2n), rem = cell - a0 * T1 * T2n;
            const int a1 = rem / T2n, a2 = rem - a1 * T2n;
            const int pl = bo.x + a0 + pad;
            if (pl < 0 || pl >= nplanes) continue;  // outside every stencil: the cell is zero
            g = ((int64_t)pl * n + wrapn(bo.y + a1, n)) * n + wrapn(bo.z + a2, n);
        } else {
            const int a0 = cell / T1, a1 = cell - a0 * T1;
            const int pl = bo.x + a0 + pad;
            if (pl < 0 || pl >= nplanes) continue;
            g = (int64_t)pl * n + wrapn(bo.y + a1, n);
        }
        atomic_add_cx(H + g, vr, vi);
    }
}

// Adds the FP64 tiles of the crowded bins into the extended spread grid (one CTA per tile).
template <typename T, int D>
__global__ void __launch_bounds__(SUB_THREADS) crowd_merge_kernel(NodeDesc nd, cx_t<T> *__restrict__ H) {
    const int ncell = (D == 3) ? nd.T[0] * nd.T[1] * nd.T[2] : nd.T[0] * nd.T[1];
    const int slot = blockIdx.x;
    const int4 bo = nd.bins[nd.crowd_bin[slot]];
    const int n = nd.n, pad = nd.pad, T1 = nd.T[1], T2n = (D == 3) ? nd.T[2] : 1;
    const int nplanes = n / 2 + 1 + 2 * pad;
    const double2 *src = nd.crowd + (int64_t)slot * ncell;
    for (int cell = threadIdx.x; cell < ncell; cell += blockDim.x) {
        const double2 v = src[cell];
        if (v.x == 0.0 && v.y == 0.0) continue;
        int64_t g;
        if (D == 3) {
            const int a0 = cell / (T1 * T2n), rem = cell - a0 * T1 * T2n;
            const int a1 = rem / T2n, a2 = rem - a1 * T2n;
            const int pl = bo.x + a0 + pad;
            if (pl < 0 || pl >= nplanes) continue;
            g = ((int64_t)pl * n + wrapn(bo.y + a1, n)) * n + wrapn(bo.z + a2, n);
        } else {
            const int a0 = cell / T1, a1 = cell - a0 * T1;
            const int pl = bo.x + a0 + pad;
            if (pl < 0 || pl >= nplanes) continue;
            g = (int64_t)pl * n + wrapn(bo.y + a1, n);
        }
        atomic_add_cx(H + g, (T)v.x, (T)v.y);
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
__global__ void __launch_bounds__(256) energy_partials_kernel(int64_t count, const T *__restrict__ u,
                                                              const T *__restrict__ rho,
                                                              double2 *__restrict__ partials) {
    __shared__ double sh[2 * 32];
    KSum acc;
    acc.init();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        acc.add((double)u[i] * (double)rho[i]);
    KSum tot = ksum_block(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(tot.s, tot.c);
}

// One CTA of 1024 threads folds the partials: thread t takes partials t, t+1024, ... in
// order, then a fixed shuffle tree combines the threads.  The result does not depend on
// timing, so repeated evaluations give identical energies.
__global__ void __launch_bounds__(1024) energy_final_kernel(const double2 *__restrict__ partials,
                                                            int nparts, double scale,
                                                            double *__restrict__ E) {
    __shared__ double sh[2 * 32];
    KSum acc;
    acc.init();
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) acc.merge(partials[q].x, partials[q].y);
    KSum tot = ksum_block(acc, sh);
    if (threadIdx.x == 0) *E = scale * tot.value();
}

// --------------------------------------------------------------------------- launchers
static inline unsigned nblk(int64_t M, int t) { return (unsigned)((M + t - 1) / t); }

template <typename T>
static cudaError_t set_smem(const void *fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
cudaError_t launch_interp(const NodeDesc &nd, const void *G, void *c_out, int apply_W,
                          cudaStream_t s) {
    if (nd.nsub == 0) return cudaSuccess;
    const size_t sm = node_smem(nd, sizeof(T) == 4 ? NLINT_FP32 : NLINT_FP64);
    cudaError_t e;
    if (nd.d == 3) {
        if ((e = set_smem<T>((const void *)interp_sub_kernel<T, 3>, sm)) != cudaSuccess) return e;
        interp_sub_kernel<T, 3><<<(unsigned)nd.nsub, SUB_THREADS, sm, s>>>(nd, (const cx_t<T> *)G, (cx_t<T> *)c_out, apply_W);
    } else {
        if ((e = set_smem<T>((const void *)interp_sub_kernel<T, 2>, sm)) != cudaSuccess) return e;
        interp_sub_kernel<T, 2><<<(unsigned)nd.nsub, SUB_THREADS, sm, s>>>(nd, (const cx_t<T> *)G, (cx_t<T> *)c_out, apply_W);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spread(const NodeDesc &nd, const void *c_in, void *Hext, cudaStream_t s) {
    if (nd.nsub == 0) return cudaSuccess;
    const size_t sm = node_smem(nd, sizeof(T) == 4 ? NLINT_FP32 : NLINT_FP64);
    cudaError_t e;
    if (nd.d == 3) {
        if ((e = set_smem<T>((const void *)spread_sub_kernel<T, 3>, sm)) != cudaSuccess) return e;
        spread_sub_kernel<T, 3><<<(unsigned)nd.nsub, SUB_THREADS, sm, s>>>(nd, (const cx_t<T> *)c_in, (cx_t<T> *)Hext);
    } else {
        if ((e = set_smem<T>((const void *)spread_sub_kernel<T, 2>, sm)) != cudaSuccess) return e;
        spread_sub_kernel<T, 2><<<(unsigned)nd.nsub, SUB_THREADS, sm, s>>>(nd, (const cx_t<T> *)c_in, (cx_t<T> *)Hext);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_crowd_merge(const NodeDesc &nd, void *Hext, cudaStream_t s) {
    if (nd.ncrowd == 0) return cudaSuccess;
    if (nd.d == 3)
        crowd_merge_kernel<T, 3><<<(unsigned)nd.ncrowd, SUB_THREADS, 0, s>>>(nd, (cx_t<T> *)Hext);
    else
        crowd_merge_kernel<T, 2><<<(unsigned)nd.ncrowd, SUB_THREADS, 0, s>>>(nd, (cx_t<T> *)Hext);
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
    energy_final_kernel<<<1, 1024, 0, s>>>(partials, nparts, scale, E);
    return cudaGetLastError();
}

#define NLINT_INST(T)                                                                              \
    template cudaError_t launch_interp<T>(const NodeDesc &, const void *, void *, int, cudaStream_t); \
    template cudaError_t launch_spread<T>(const NodeDesc &, const void *, void *, cudaStream_t);      \
    template cudaError_t launch_crowd_merge<T>(const NodeDesc &, void *, cudaStream_t);              \
    template cudaError_t launch_scatter_canonical<T>(int64_t, const void *, const int32_t *,         \
                                                     const int32_t *, double, void *, cudaStream_t); \
    template cudaError_t launch_gather_canonical<T>(int64_t, const void *, const int32_t *,          \
                                                    const int32_t *, void *, cudaStream_t);          \
    template cudaError_t launch_energy_partials<T>(int64_t, const void *, const void *, double2 *,   \
                                                   int, cudaStream_t);
NLINT_INST(float)
NLINT_INST(double)

}  // namespace nlint
