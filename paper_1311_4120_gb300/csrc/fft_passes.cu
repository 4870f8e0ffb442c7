// Oversampled-grid FFT passes (eq. fft, Section 2; steps a1/a2 and a6/a7 of the path).
//
// A pass transforms all lines along one axis.  Each CTA stages a tile of lines in shared
// memory (lines as columns of an [n][LD] array), runs a mixed-radix Stockham transform
// (radix 8/4/2/3) in place with one barrier between the reads and the writes of each stage,
// and writes the tile back.  Loading and storing apply the pass's pruning:
//   * mode-centred inputs: only the N nonzero entries (modes m in [-N/2, N/2), placed at
//     fine index m mod n) are read, the rest of the line is zero;
//   * Hermitian inputs: only n/2+1 entries are read; the rest follow by conjugate symmetry;
//   * half / mode outputs: only the entries later stages use are written.
// The first forward pass multiplies the density by the deconvolution product (type-2
// pre-correction) and the last inverse pass applies the type-1 post-correction, takes the
// real part and accumulates the energy sum (Remark 3.3) in FP64 with compensation.
#include "common.cuh"
#include "internal.h"

namespace nlint {

// Butterflies held per thread per stage, by radix.  With TPC = ceil(n/16) threads per
// line every radix-8/4/2 stage fits exactly and a radix-3 stage needs at most 6.
template <int R> struct MaxB;
template <> struct MaxB<8> { static constexpr int v = 2; };
template <> struct MaxB<4> { static constexpr int v = 4; };
template <> struct MaxB<2> { static constexpr int v = 8; };
template <> struct MaxB<3> { static constexpr int v = 6; };

template <typename T, int R>
__device__ __forceinline__ void dft_small(cx_t<T> *v, int sign) {
    using T2 = cx_t<T>;
    if constexpr (R == 2) {
        T2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 3) {
        const T c = T(-0.5);
        const T s = T(sign) * T(0.86602540378443864676);  // sign * sqrt(3)/2
        T2 a = v[0], b = v[1], d = v[2];
        T2 sum = cadd(b, d), dif = csub(b, d);
        T2 m = cadd(a, cscale(sum, c));
        T2 rot = cmake<T2>(-s * dif.y, s * dif.x);     // i s (b - d)
        v[0] = cadd(a, sum);
        v[1] = cadd(m, rot);
        v[2] = csub(m, rot);
    } else if constexpr (R == 4) {
        T2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        T2 t2 = cadd(v[1], v[3]), t3 = cmuli(csub(v[1], v[3]), sign);
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    } else if constexpr (R == 8) {
        T2 e[4] = {v[0], v[2], v[4], v[6]};
        T2 o[4] = {v[1], v[3], v[5], v[7]};
        dft_small<T, 4>(e, sign);
        dft_small<T, 4>(o, sign);
        const T h = T(0.70710678118654752440);
        // W8^k = exp(sign i pi k / 4)
        T2 o1 = cmul(o[1], cmake<T2>(h, T(sign) * h));
        T2 o2 = cmuli(o[2], sign);
        T2 o3 = cmul(o[3], cmake<T2>(-h, T(sign) * h));
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
}

// One Stockham stage of radix R on every column of buf ([n][LD], column `col`).
// p = product of the radices already applied; tw[q] = exp(-2 pi i q / n).
template <typename T, int R>
__device__ __forceinline__ void fft_stage(cx_t<T> *buf, int n, int LD, int col, int tc, int TPC,
                                          int p, const cx_t<T> *__restrict__ tw, int sign) {
    using T2 = cx_t<T>;
    constexpr int MB = MaxB<R>::v;
    const int nb = (tc < TPC) ? n / R : 0;  // threads past TPC (warp padding) only sync
    T2 v[MB][R];
#pragma unroll
    for (int b = 0; b < MB; b++) {
        const int i = tc + b * TPC;
        if (i < nb) {
#pragma unroll
            for (int r = 0; r < R; r++) v[b][r] = buf[(i + r * nb) * LD + col];
        }
    }
    __syncthreads();
    const int step = n / (p * R);
#pragma unroll
    for (int b = 0; b < MB; b++) {
        const int i = tc + b * TPC;
        if (i < nb) {
            const int k = i % p;
#pragma unroll
            for (int r = 1; r < R; r++) {
                T2 w = tw[r * k * step];
                if (sign > 0) w = cconj(w);
                v[b][r] = cmul(v[b][r], w);
            }
            dft_small<T, R>(v[b], sign);
            const int j = (i - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; r++) buf[(j + r * p) * LD + col] = v[b][r];
        }
    }
    __syncthreads();
}

// Radix sequences are 8...8 [4] [2] 3...3 (see make_radix), so each stage kind appears once.
template <typename T>
__device__ __forceinline__ void fft_columns(cx_t<T> *buf, const PassDesc &p, int col, int tc,
                                            const cx_t<T> *__restrict__ tw) {
    int pp = 1, s = 0;
    for (; s < p.nrad && p.rad[s] == 8; s++, pp *= 8)
        fft_stage<T, 8>(buf, p.n, p.LD, col, tc, p.TPC, pp, tw, p.sign);
    if (s < p.nrad && p.rad[s] == 4) {
        fft_stage<T, 4>(buf, p.n, p.LD, col, tc, p.TPC, pp, tw, p.sign);
        pp *= 4;
        s++;
    }
    if (s < p.nrad && p.rad[s] == 2) {
        fft_stage<T, 2>(buf, p.n, p.LD, col, tc, p.TPC, pp, tw, p.sign);
        pp *= 2;
        s++;
    }
    for (; s < p.nrad; s++, pp *= 3)
        fft_stage<T, 3>(buf, p.n, p.LD, col, tc, p.TPC, pp, tw, p.sign);
}

// CTA reduction of the compensated energy sums; thread 0 writes the CTA's partial.
__device__ __forceinline__ void block_reduce_ksum(KSum acc, double2 *out, void *scratch) {
    KSum tot = ksum_block(acc, reinterpret_cast<double *>(scratch));
    if (threadIdx.x == 0) *out = make_double2(tot.s, tot.c);
}

// --------------------------------------------------------------------------- column pass
template <typename T>
__global__ void __launch_bounds__(256) colpass_kernel(PassDesc p, const void *__restrict__ vin,
                                                      void *__restrict__ vout,
                                                      const cx_t<T> *__restrict__ tw) {
    using T2 = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *buf = reinterpret_cast<T2 *>(smem_raw);
    const int64_t tiles = (p.I + p.B - 1) / p.B;
    const int64_t o = blockIdx.x / tiles;
    const int64_t i = (blockIdx.x % tiles) * p.B + (threadIdx.x % p.B);
    const int col = threadIdx.x % p.B, tc = threadIdx.x / p.B;
    const bool valid = (tc < p.TPC) && (i < p.I);
    const int n = p.n, N = p.N, h = N / 2;
    const T *fac = reinterpret_cast<const T *>(p.fac);

    T bfac = T(1);
    if (valid && (p.in_kind == IN_REAL_MODES || p.out_kind == OUT_REAL_MODES))
        bfac = (p.dim == 3) ? fac[i / N] * fac[i % N] : fac[i];

    if (tc < p.TPC) {
        for (int r = tc; r < n; r += p.TPC) {
            T2 v = czero<T2>();
            if (valid) {
                if (p.in_kind == IN_REAL_MODES || p.in_kind == IN_CPLX_MODES) {
                    const int m = (r < n / 2) ? r : r - n;
                    if (m >= -h && m < h) {
                        const int a = m + h;
                        const int64_t idx = o * p.in_so + (int64_t)a * p.in_sa + i;
                        if (p.in_kind == IN_REAL_MODES) {
                            v.x = reinterpret_cast<const T *>(vin)[idx] * fac[a] * bfac;
                        } else {
                            v = reinterpret_cast<const T2 *>(vin)[idx];
                        }
                    }
                } else if (p.in_kind == IN_CPLX_FULL) {
                    v = reinterpret_cast<const T2 *>(vin)[o * p.in_so + (int64_t)r * p.in_sa + i];
                } else {  // IN_CPLX_HERM
                    if (r <= n / 2) v = reinterpret_cast<const T2 *>(vin)[o * p.in_so + (int64_t)r * p.in_sa + i];
                    else v = cconj(reinterpret_cast<const T2 *>(vin)[o * p.in_so + (int64_t)(n - r) * p.in_sa + i]);
                }
            }
            buf[r * p.LD + col] = v;
        }
    }
    __syncthreads();
    fft_columns<T>(buf, p, col, tc, tw);

    KSum acc;
    acc.init();
    if (valid) {
        if (p.out_kind == OUT_CPLX_FULL || p.out_kind == OUT_CPLX_HALF) {
            const int rows = (p.out_kind == OUT_CPLX_FULL) ? n : n / 2 + 1;
            for (int r = tc; r < rows; r += p.TPC)
                reinterpret_cast<T2 *>(vout)[o * p.out_so + (int64_t)r * p.out_sa + i] = buf[r * p.LD + col];
        } else if (p.out_kind == OUT_CPLX_MODES) {
            for (int a = tc; a < N; a += p.TPC) {
                const int r = (a - h + n) % n;
                reinterpret_cast<T2 *>(vout)[o * p.out_so + (int64_t)a * p.out_sa + i] = buf[r * p.LD + col];
            }
        } else {  // OUT_REAL_MODES (+ energy)
            const T *rho = reinterpret_cast<const T *>(p.rho);
            for (int a = tc; a < N; a += p.TPC) {
                const int r = (a - h + n) % n;
                const int64_t idx = o * p.out_so + (int64_t)a * p.out_sa + i;
                const T val = buf[r * p.LD + col].x * fac[a] * bfac;
                reinterpret_cast<T *>(vout)[idx] = val;
                if (rho) acc.add((double)val * (double)rho[idx]);
            }
        }
    }
    if (p.out_kind == OUT_REAL_MODES && p.partials) block_reduce_ksum(acc, p.partials + blockIdx.x, smem_raw);
}

// --------------------------------------------------------------------------- row pass
// Lines are contiguous rows q = 0..I-1 (input row stride in_so, output row stride out_so).
// IN_CPLX_FOLD reads the spread grid H+ of the half node set, stored on the slowest axis
// at planes lz = -pad .. n/2+pad (plane lz at storage plane lz + pad), and forms the
// Hermitian grid H[l] = H+[l] + conj(H+[-l]) for the stored half lz in [0, n/2].
template <typename T>
__global__ void __launch_bounds__(256) rowpass_kernel(PassDesc p, const void *__restrict__ vin,
                                                      void *__restrict__ vout,
                                                      const cx_t<T> *__restrict__ tw) {
    using T2 = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *buf = reinterpret_cast<T2 *>(smem_raw);
    const int n = p.n, N = p.N, h = N / 2;
    const int64_t q0 = (int64_t)blockIdx.x * p.B;
    const T2 *in = reinterpret_cast<const T2 *>(vin);
    T2 *out = reinterpret_cast<T2 *>(vout);
    const int nthr = p.B * p.TPC;  // threads past nthr (warp padding) only take part in syncs

    for (int idx = threadIdx.x; idx < p.B * n && threadIdx.x < nthr; idx += nthr) {
        const int row = idx / n, r = idx % n;
        const int64_t q = q0 + row;
        T2 v = czero<T2>();
        if (q < p.I) {
            if (p.in_kind == IN_CPLX_MODES) {
                const int m = (r < n / 2) ? r : r - n;
                if (m >= -h && m < h) v = in[q * p.in_so + (m + h)];
            } else if (p.in_kind == IN_CPLX_FULL) {
                v = in[q * p.in_so + r];
            } else {  // IN_CPLX_FOLD
                const int64_t lz = q / p.fold_rows_per_plane, ly = q % p.fold_rows_per_plane;
                v = in[(lz + p.fold_pad) * p.fold_plane + ly * n + r];
                int64_t mz = INT64_MIN;
                if (lz <= p.fold_pad) mz = -lz;
                else if (lz >= n / 2 - p.fold_pad) mz = n - lz;
                if (mz != INT64_MIN) {
                    const int64_t my = (p.fold_rows_per_plane == 1) ? 0 : (n - ly) % n;
                    const int rr = (n - r) % n;
                    v = cadd(v, cconj(in[(mz + p.fold_pad) * p.fold_plane + my * n + rr]));
                }
            }
        }
        buf[r * p.LD + row] = v;
    }
    __syncthreads();
    const int col = threadIdx.x % p.B, tc = threadIdx.x / p.B;
    fft_columns<T>(buf, p, col, tc, tw);

    const int out_len = (p.out_kind == OUT_CPLX_MODES) ? N : n;
    for (int idx = threadIdx.x; idx < p.B * out_len && threadIdx.x < nthr; idx += nthr) {
        const int row = idx / out_len, a = idx % out_len;
        const int64_t q = q0 + row;
        if (q >= p.I) continue;
        const int r = (p.out_kind == OUT_CPLX_MODES) ? (a - h + n) % n : a;
        out[q * p.out_so + a] = buf[r * p.LD + row];
    }
}

// --------------------------------------------------------------------------- host side
void make_radix(int n, PassDesc &p) {
    int m = n, k = 0;
    while (m % 8 == 0 && m > 1 && k < 12) { p.rad[k++] = 8; m /= 8; }
    if (m % 4 == 0 && k < 12) { p.rad[k++] = 4; m /= 4; }
    if (m % 2 == 0 && k < 12) { p.rad[k++] = 2; m /= 2; }
    while (m % 3 == 0 && m > 1 && k < 12) { p.rad[k++] = 3; m /= 3; }
    p.nrad = (m == 1) ? k : -1;
}

void config_pass(PassDesc &p, int prec, bool row) {
    const int target = (prec == NLINT_FP32) ? 256 : 128;
    p.TPC = (p.n + 15) / 16;
    p.B = target / p.TPC;
    if (p.B < 1) p.B = 1;
    if (!row && p.B > p.I) p.B = (int)p.I;
    if (row && p.B > p.I) p.B = (int)p.I;
    p.LD = row ? (p.B | 1) : p.B;
}

bool pass_fits(const PassDesc &p) {
    for (int s = 0; s < p.nrad; s++) {
        const int R = p.rad[s];
        const int mb = R == 8 ? 2 : R == 4 ? 4 : R == 2 ? 8 : 6;
        const int nb = p.n / R;
        if ((nb + p.TPC - 1) / p.TPC > mb) return false;
    }
    return p.nrad > 0 && pass_threads(p) <= 256;  // the kernels are compiled for <= 256 threads
}

// Threads per CTA: B lines x TPC threads, rounded up to whole warps.
int pass_threads(const PassDesc &p) { return (p.B * p.TPC + 31) / 32 * 32; }

int64_t pass_blocks(const PassDesc &p, bool row) {
    if (row) return (p.I + p.B - 1) / p.B;
    return p.n_outer * ((p.I + p.B - 1) / p.B);
}

size_t pass_smem(const PassDesc &p, int prec) {
    const size_t cs = (prec == NLINT_FP32) ? 8 : 16;
    size_t s = (size_t)p.n * p.LD * cs;
    const size_t red = 64 * sizeof(double);  // energy reduction scratch (2 doubles per warp)
    return s > red ? s : red;
}

template <typename T>
cudaError_t launch_colpass(const PassDesc &p, const void *in, void *out, const void *tw,
                           cudaStream_t s) {
    const int prec = sizeof(T) == 4 ? NLINT_FP32 : NLINT_FP64;
    const size_t smem = pass_smem(p, prec);
    cudaError_t e = cudaFuncSetAttribute(colpass_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t nb = pass_blocks(p, false);
    colpass_kernel<T><<<(unsigned)nb, pass_threads(p), smem, s>>>(p, in, out, reinterpret_cast<const cx_t<T> *>(tw));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rowpass(const PassDesc &p, const void *in, void *out, const void *tw,
                           cudaStream_t s) {
    const int prec = sizeof(T) == 4 ? NLINT_FP32 : NLINT_FP64;
    const size_t smem = pass_smem(p, prec);
    cudaError_t e = cudaFuncSetAttribute(rowpass_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t nb = pass_blocks(p, true);
    rowpass_kernel<T><<<(unsigned)nb, pass_threads(p), smem, s>>>(p, in, out, reinterpret_cast<const cx_t<T> *>(tw));
    return cudaGetLastError();
}

template cudaError_t launch_colpass<float>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
template cudaError_t launch_colpass<double>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
template cudaError_t launch_rowpass<float>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
template cudaError_t launch_rowpass<double>(const PassDesc &, const void *, void *, const void *, cudaStream_t);

}  // namespace nlint
