// Oversampled-grid FFT passes (eq. fft; steps a1/a2 and a6/a7/a8 of the path).
//
// A pass transforms every line along one axis of a 2D/3D array with one HBM read and one HBM
// write.  The FFT length n is a template parameter (n = 2^a or 3*2^a, 16..2048), so the radix
// schedule (radix 8 stages, then one radix 4 or 2, then one radix 3) and every stride are
// compile-time constants.  Each thread owns VPT values of its line per stage: the first stage
// reads its butterflies straight from global memory (coalesced across the lines of the CTA
// in a column pass, along the line in a row pass), the middle stages exchange through shared
// memory (Stockham autosort), and the last stage writes straight to global memory.
//
// Pruning: mode-centred inputs read only the N nonzero entries (mode m at FFT index m mod n);
// Hermitian inputs read n/2+1 entries and form the rest by conjugate symmetry; half and mode
// outputs write only the entries later stages use.  The first forward pass multiplies the
// density by the deconvolution product (type-2 pre-correction); the last inverse pass applies
// the type-1 post-correction, takes the real part and adds u*rho into an FP64 energy partial
// per CTA (Remark 3.3).
#pragma once
#include "common.cuh"
#include "internal.h"

namespace nlint {

// ------------------------------------------------------------------ compile-time schedule
// Schedule 0: radix 8 stages, then one radix 4 or 2, then one radix 3.  Schedule 1 (lines of 2^a
// points, a >= 7; chosen per plan and pass class, nlint_params.fft_sched): two stages of radix
// 2^ceil(a/2) and 2^floor(a/2) (a <= 10; a = 11: 16, 16, 8), so that a line takes one exchange
// through shared memory instead of two, with each thread holding one or two whole butterflies
// of the larger radix.
__host__ __device__ constexpr bool fft_has3(int n) { return n % 3 == 0; }
__host__ __device__ constexpr int fft_log2(int m) { return m <= 1 ? 0 : 1 + fft_log2(m / 2); }
__host__ __device__ constexpr bool fft_two_stage(int n, int v) { return v && !fft_has3(n) && n >= 128; }
__host__ __device__ constexpr int fft_pow2(int n) { return fft_log2(fft_has3(n) ? n / 3 : n); }
__host__ __device__ constexpr int fft_eights(int n) { return fft_pow2(n) / 3; }
__host__ __device__ constexpr int fft_tail(int n) {  // 4, 2 or 1 after the radix-8 stages
    return fft_pow2(n) % 3 == 2 ? 4 : (fft_pow2(n) % 3 == 1 ? 2 : 1);
}
__host__ __device__ constexpr int fft_nstages(int n, int v = 0) {
    return fft_two_stage(n, v) ? (fft_log2(n) <= 10 ? 2 : 3)
                               : fft_eights(n) + (fft_tail(n) > 1 ? 1 : 0) + (fft_has3(n) ? 1 : 0);
}
__host__ __device__ constexpr int fft_radix(int n, int s, int v = 0) {
    return fft_two_stage(n, v)
               ? (fft_log2(n) <= 10 ? (s == 0 ? 1 << ((fft_log2(n) + 1) / 2) : 1 << (fft_log2(n) / 2))
                                    : (s < 2 ? 16 : 8))
               : (s < fft_eights(n) ? 8 : (s == fft_eights(n) && fft_tail(n) > 1) ? fft_tail(n) : 3);
}
__host__ __device__ constexpr int fft_pprod(int n, int s, int v = 0) {  // product of the radices before s
    return s == 0 ? 1 : fft_pprod(n, s - 1, v) * fft_radix(n, s - 1, v);
}
// Pass modes: 0 column pass; 1 row pass; 2 row pass that reads more than it writes (the fold
// input of the first inverse pass), which wants more threads per line.
// Tuning constants for 2^a lines of n <= 512, per pass mode: values per thread, and the
// resident CTAs that FP32 launches of 512 threads (mode 5: any size) ask for (0: the
// compiler's choice).  Chosen by CUDA-event timing of each pass on the 3D 256^3 workload
// (512^3 fine grid, FP32): the values per thread that gave the shortest pass per mode.
constexpr int FFT_VPT0 = 16, FFT_MINB0 = 0;                 // column passes
constexpr int FFT_VPT1 = 16, FFT_MINB1 = 0;                 // row passes
// packed real-data column passes: four resident CTAs of 512 threads cap them at 32 registers
// (40-76 bytes of spills at n = 512) and still measured faster than three (forward 0.094 ->
// 0.087 ms, inverse 0.156 -> 0.133 ms at n = 512): these passes are bound by load latency
constexpr int FFT_PACKED_VPT = 8, FFT_PACKED_MINB = 4;
constexpr int FFT_DUAL_VPT = 16, FFT_DUAL_MINB = 3;         // dual column passes (modes 6, 7)
constexpr int FFT_STAGED_MINB = 4;  // packed passes with staged input (kernel variant 2)
__host__ __device__ constexpr int fft_vpt_small(int mode) {
    return mode == 0 ? FFT_VPT0 : mode == 1 ? FFT_VPT1 : mode == 2 ? 8
         : (mode == 3 || mode == 4) ? FFT_PACKED_VPT : (mode == 6 || mode == 7) ? FFT_DUAL_VPT : 16;
}
// Schedule 1 (the two-stage radix schedule above) for modes 0-4 on lines of 2^a >= 128 points:
// each thread holds the larger radix's worth of values (16 or 32).  3 * 2^a lines, shorter lines
// and modes 5-7 have schedule 0 only.
__host__ __device__ constexpr bool fft_has_alt(int n, int mode) { return fft_two_stage(n, 1) && mode <= 4; }
__host__ __device__ constexpr int fft_vpt(int n, int mode = 0, int v = 0) {
    return (v && fft_has_alt(n, mode)) ? fft_radix(n, 0, 1)
                                       : (fft_has3(n) ? 24 : (n <= 512 ? fft_vpt_small(mode) : 32));
}
__host__ __device__ constexpr int fft_vpt_ref(int n) { return fft_has3(n) ? 24 : (n <= 512 ? 16 : 32); }
__host__ __device__ constexpr int fft_tpl(int n, int mode = 0, int v = 0) { return n / fft_vpt(n, mode, v); }  // 2^k
// padded row line: one pad cell per 16 (schedule 0) or per radix of the first stage (schedule 1,
// whose first stage writes each thread's butterfly as a run of that many cells)
__host__ __device__ constexpr int fft_row_ld(int n, int v = 0) {
    return fft_two_stage(n, v) ? n + n / fft_radix(n, 0, 1) : n + n / 16;
}
// Lines per CTA.  Column pass: 128-byte rows (16 FP32 / 8 FP64 complex), fewer for the
// longest lines (shared memory <= 192 KB), at least one warp.
// Row pass: about 512 threads, at most 96 KB of shared memory, whole warps where possible.
__host__ __device__ constexpr int fft_pow2_floor(int m) { return m < 2 ? 1 : 2 * fft_pow2_floor(m / 2); }
__host__ __device__ constexpr int fft_col_b_raw(int n, int cs) {  // <= 192 KB of shared memory
    return (128 / cs) < fft_pow2_floor(196608 / (n * cs)) ? 128 / cs : fft_pow2_floor(196608 / (n * cs));
}
__host__ __device__ constexpr int fft_col_b(int n, int cs) {  // at the reference 16 values
    return fft_col_b_raw(n, cs) * (n / fft_vpt_ref(n)) >= 32 ? fft_col_b_raw(n, cs) : 32 / (n / fft_vpt_ref(n));
}
// per mode: column passes with half the values per thread take half the lines per CTA
__host__ __device__ constexpr int fft_col_b_m(int n, int cs, int mode, int v = 0) {
    return (fft_vpt(n, mode, v) * 2 == fft_vpt_ref(n) && fft_col_b(n, cs) >= 2) ? fft_col_b(n, cs) / 2
                                                                                : fft_col_b(n, cs);
}
// Row pass: about 256 threads (mode 1, and every schedule-1 pass) or 512 threads (mode 2) per CTA.
__host__ __device__ constexpr int fft_row_thr(int mode, int v = 0) { return (mode == 2 && !v) ? 512 : 256; }
__host__ __device__ constexpr int fft_row_b_raw(int n, int cs, int mode, int v = 0) {
    return (fft_row_thr(mode, v) / fft_tpl(n, mode, v)) < (96 * 1024) / (fft_row_ld(n, v) * cs)
               ? fft_row_thr(mode, v) / fft_tpl(n, mode, v)
               : (96 * 1024) / (fft_row_ld(n, v) * cs);
}
__host__ __device__ constexpr int fft_row_b(int n, int cs, int mode = 1, int v = 0) {
    return fft_row_b_raw(n, cs, mode, v) < 1 ? 1
         : (fft_tpl(n, mode, v) < 32 && fft_row_b_raw(n, cs, mode, v) >= 32 / fft_tpl(n, mode, v))
               ? fft_row_b_raw(n, cs, mode, v) / (32 / fft_tpl(n, mode, v)) * (32 / fft_tpl(n, mode, v))
               : fft_row_b_raw(n, cs, mode, v);
}

// Modes 3 and 4 are column passes that carry two real lines per complex FFT line: mode 3
// transforms real input to the Hermitian half (z = x + i y, then X, Y from Z(k) and Z(n-k)),
// mode 4 the Hermitian half back to real output (Z = X + i Y, then x = Re z, y = Im z).
// Mode 5 is a row pass that convolves each line: forward FFT, times a real row of `mult`,
// inverse FFT (the multiply of an FFT convolution fused between two transforms of one axis).
__host__ __device__ constexpr bool fft_is_row(int mode) { return mode == 1 || mode == 2 || mode == 5; }
__host__ __device__ constexpr bool fft_packed(int mode) { return mode == 3 || mode == 4; }
// Modes 6 and 7: the dual column passes of Algorithm 2 along z.  6: one real input line carried
// twice, with the unit factors (I_1) and with the deconvolution factors `fac2` (I_2), as
// z = x1 + i x2; the half (k <= n/2) of X1 goes to the output, the window (k <= win) of X2 to
// `out2`.  7: the Hermitian half of I_1 (input) and the window half of I_2 (`in2`) as
// Z = X1 + i X2; the output is Re z (unit factors) + Im z times the deconvolution (+ energy).
__host__ __device__ constexpr bool fft_dual(int mode) { return mode == 6 || mode == 7; }
__host__ __device__ constexpr int fft_pack(int mode) { return fft_packed(mode) ? 2 : 1; }

// Kernel variant 2 of the FP32 packed real-data passes (modes 3, 4; the geometry of schedule 0):
// the CTA's input is staged in shared memory by 16-byte asynchronous copies (cp.async) before
// the first stage.  Used whenever the rows of a CTA's data columns are 16-byte aligned runs
// (fft_stage_ok): at four resident CTAs the register loads of schedule 0 (32 registers per
// thread) cannot hold a line's loads in flight, while the copies need no registers.  Rows
// staged: mode 3 the N real modes of each column, mode 4 the Hermitian half (entries 0..n/2,
// or 0..win within a window); elements of 4 (mode 3) or 8 (mode 4) bytes.
__host__ __device__ constexpr bool fft_stages_input(int mode, int v, int cs) {
    return (mode == 3 || mode == 4) && v == 2 && cs == 8;
}
__host__ __device__ constexpr int fft_stage_rows(int mode, int n, int N, int win) {
    return mode == 3 ? N : ((win > 0 && win < n / 2) ? win + 1 : n / 2 + 1);
}

// Input and output kinds each mode is launched with (compile-time, so a single-kind mode has no
// branch on the kind; the launcher rejects anything else).
__host__ __device__ constexpr unsigned fft_in_mask(int mode) {
    return mode == 0 ? (1u << IN_CPLX_MODES) | (1u << IN_CPLX_FULL) | (1u << IN_CPLX_WIN)
         : mode == 2 ? (1u << IN_CPLX_FOLD)
         : (mode == 3 || mode == 6) ? (1u << IN_REAL_MODES)
         : (mode == 4 || mode == 7) ? (1u << IN_CPLX_HERM)
                     : (1u << IN_CPLX_MODES);  // 1, 5
}
__host__ __device__ constexpr unsigned fft_out_mask(int mode) {
    return mode == 0 ? (1u << OUT_CPLX_FULL) | (1u << OUT_CPLX_MODES) | (1u << OUT_CPLX_WIN)
         : mode == 1 ? (1u << OUT_CPLX_FULL)
         : (mode == 3 || mode == 6) ? (1u << OUT_CPLX_HALF)
         : (mode == 4 || mode == 7) ? (1u << OUT_REAL_MODES)
                     : (1u << OUT_CPLX_MODES);  // 2, 5
}

template <typename T, int NF, int MODE, int V = 0>
struct FftCfg {
    static constexpr int CS = (int)(2 * sizeof(T));
    static constexpr int VG = V == 1 ? 1 : 0;  // the schedule that sets the geometry
    static constexpr int TPL = fft_tpl(NF, MODE, VG);  // threads per line
    static constexpr int NST = fft_nstages(NF, VG);
    static constexpr int B = fft_is_row(MODE) ? fft_row_b(NF, CS, MODE, VG) : fft_col_b_m(NF, CS, MODE, VG);  // lines
    static constexpr int ROW_LD = fft_row_ld(NF, VG);
    // row passes: shared index of line entry e, one pad cell per 2^PADSH entries
    static constexpr int PADSH = fft_two_stage(NF, VG) ? fft_log2(fft_radix(NF, 0, 1)) : 4;
    static constexpr int THREADS = B * TPL;
    // packed passes hold two lines' loads in flight: ask for two resident CTAs of 512 threads
    static constexpr bool F32_512 = THREADS == 512 && NF <= 512 && sizeof(T) == 4 && V == 0;
    static constexpr int MIN_BLOCKS = (V == 2 && THREADS == 512 && NF <= 512) ? FFT_STAGED_MINB
                                    : (fft_packed(MODE) && F32_512) ? FFT_PACKED_MINB
                                    : (fft_dual(MODE) && F32_512) ? FFT_DUAL_MINB
                                    : (MODE == 0 && F32_512) ? FFT_MINB0
                                    : (MODE == 1 && F32_512) ? FFT_MINB1
                                    : (MODE == 5 && NF <= 512 && sizeof(T) == 4 && V == 0) ? 3 : 0;
};

// ------------------------------------------------------------------ butterflies
// cos and sin of 2 pi m / R at compile time (R a multiple of 4): the quadrant is taken out
// exactly, the rest (below pi / 2) by Taylor series to double precision
__host__ __device__ constexpr double ct_sin_q(double x) {
    double t = x, s = x;
    for (int k = 1; k < 14; k++) {
        t *= -x * x / (double)((2 * k) * (2 * k + 1));
        s += t;
    }
    return s;
}
__host__ __device__ constexpr double ct_cos_q(double x) {
    double t = 1.0, s = 1.0;
    for (int k = 1; k < 14; k++) {
        t *= -x * x / (double)((2 * k - 1) * (2 * k));
        s += t;
    }
    return s;
}
__host__ __device__ constexpr double ct_cos2pi(int m, int R) {
    const int q = (4 * (m % R)) / R;
    const double ph = 6.283185307179586476925286766559 * (double)((m % R) - q * (R / 4)) / (double)R;
    return q == 0 ? ct_cos_q(ph) : q == 1 ? -ct_sin_q(ph) : q == 2 ? -ct_cos_q(ph) : ct_sin_q(ph);
}
__host__ __device__ constexpr double ct_sin2pi(int m, int R) {
    const int q = (4 * (m % R)) / R;
    const double ph = 6.283185307179586476925286766559 * (double)((m % R) - q * (R / 4)) / (double)R;
    return q == 0 ? ct_sin_q(ph) : q == 1 ? ct_cos_q(ph) : q == 2 ? -ct_sin_q(ph) : -ct_cos_q(ph);
}

template <typename T, int R>
__device__ __forceinline__ void dft_small(cx_t<T> *v, int sign);

// DFT of R = P Q points in registers (Cooley-Tukey, input index j1 + P j2, output k1 + Q k2):
// Q-point DFTs over j2, twiddles W_R^(j1 k1) (compile-time constants), P-point DFTs over j1
template <typename T, int P, int Q>
__device__ __forceinline__ void dft_split(cx_t<T> *v, int sign) {
    using T2 = cx_t<T>;
    constexpr int R = P * Q;
    T2 y[P][Q];
#pragma unroll
    for (int j1 = 0; j1 < P; j1++) {
#pragma unroll
        for (int j2 = 0; j2 < Q; j2++) y[j1][j2] = v[j1 + P * j2];
        dft_small<T, Q>(y[j1], sign);
    }
    static_for<1, P>([&](auto J1) {
        static_for<1, Q>([&](auto K1) {
            constexpr int j1 = decltype(J1)::value, k1 = decltype(K1)::value, m = (j1 * k1) % R;
            constexpr T c = (T)ct_cos2pi(m, R), sn = (T)ct_sin2pi(m, R);
            y[j1][k1] = cmul(y[j1][k1], cmake<T2>(c, T(sign) * sn));
        });
    });
#pragma unroll
    for (int k1 = 0; k1 < Q; k1++) {
        T2 x[P];
#pragma unroll
        for (int j1 = 0; j1 < P; j1++) x[j1] = y[j1][k1];
        dft_small<T, P>(x, sign);
#pragma unroll
        for (int k2 = 0; k2 < P; k2++) v[k1 + Q * k2] = x[k2];
    }
}

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
        T2 rot = cmake<T2>(-s * dif.y, s * dif.x);  // i s (b - d)
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
        T2 o1 = cmul(o[1], cmake<T2>(h, T(sign) * h));  // W8^k = exp(sign i pi k / 4)
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
    } else if constexpr (R == 16) {
        dft_split<T, 4, 4>(v, sign);
    } else if constexpr (R == 32) {
        dft_split<T, 8, 4>(v, sign);
    }
}

// ------------------------------------------------------------------ line input
// Per-line context: where its input and output live and how its entries map to FFT indices.
template <typename T>
struct LineIO {
    using T2 = cx_t<T>;
    int n, h, kind;
    const T *fac;
    bool valid;
    int64_t in_base, out_base;  // element offsets of entry 0
    int64_t in_st, out_st;      // element stride along the line
    T bfac;                     // deconvolution product over the other axes
    int64_t mirror_base;        // fold: the mirrored line of H+, or -1
    int win;                    // frequency window (0 = none), see PassDesc

    // FFT-index entry e of the input line (zero outside the stored modes); KM: the kinds the
    // calling pass can have (one kind: no test of `kind` at all)
    template <unsigned KM>
    __device__ __forceinline__ T2 load(int e, const void *vin) const {
        constexpr bool ONE = (KM & (KM - 1)) == 0;
        auto is = [&](int k) { return (KM & (1u << k)) != 0 && (ONE || kind == k); };
        T2 v = czero<T2>();
        if (!valid) return v;
        if (is(IN_REAL_MODES) || is(IN_CPLX_MODES)) {
            const int m = e < n / 2 ? e : e - n;
            if (m >= -h && m < h) {
                const int a = m + h;
                if (is(IN_REAL_MODES)) {
                    v.x = reinterpret_cast<const T *>(vin)[in_base + a * in_st] * fac[a] * bfac;
                } else {
                    v = reinterpret_cast<const T2 *>(vin)[in_base + a * in_st];
                }
            }
        } else if (is(IN_CPLX_FULL)) {
            v = reinterpret_cast<const T2 *>(vin)[in_base + e * in_st];
        } else if (is(IN_CPLX_HERM)) {
            if (win > 0 && (e <= n / 2 ? e : n - e) > win) return v;  // outside the window
            v = (e <= n / 2) ? reinterpret_cast<const T2 *>(vin)[in_base + e * in_st]
                             : cconj(reinterpret_cast<const T2 *>(vin)[in_base + (n - e) * in_st]);
        } else if (is(IN_CPLX_WIN)) {
            const int c = e <= win ? e : (e >= n - win ? e - n + 2 * win + 1 : -1);
            if (c >= 0) v = reinterpret_cast<const T2 *>(vin)[in_base + c * in_st];
        } else if (is(IN_CPLX_FOLD)) {  // H[l] = H+[l] + conj(H+[-l])
            const T2 *in = reinterpret_cast<const T2 *>(vin);
            v = in[in_base + e];
            if (mirror_base >= 0) v = cadd(v, cconj(in[mirror_base + (e == 0 ? 0 : n - e)]));
        }
        return v;
    }
};

// ------------------------------------------------------------------ the pass kernel
// MODE 0: column pass, the CTA's B lines are adjacent in memory (128-byte rows);
// MODE 1, 2: row pass, each line is contiguous (B lines per CTA);
// MODE 3, 4: column pass with two data columns per FFT line (2B adjacent columns per CTA);
// MODE 6, 7: column pass with two transforms of one data column per FFT line (B columns).
template <typename T, int NF, int MODE, int V>
__global__ void __launch_bounds__(FftCfg<T, NF, MODE, V>::THREADS, FftCfg<T, NF, MODE, V>::MIN_BLOCKS) fft_pass_kernel(
    PassDesc P, const void *__restrict__ vin, void *__restrict__ vout, const cx_t<T> *__restrict__ tw) {
    pdl_wait();  // (launched by launch_pdl)
    pdl_trigger();
    using T2 = cx_t<T>;
    using C = FftCfg<T, NF, MODE, V>;
    constexpr bool ROW = fft_is_row(MODE);
    constexpr bool PACK = fft_packed(MODE);
    constexpr bool DUAL = fft_dual(MODE);
    constexpr bool NATURAL = PACK || DUAL;  // last stage leaves z in natural order for an epilogue
    constexpr int B = C::B;
    constexpr int TPL = C::TPL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *buf = reinterpret_cast<T2 *>(smem_raw);

    const int ll = ROW ? (int)threadIdx.x / TPL : (int)threadIdx.x % B;  // line within the CTA
    const int t = ROW ? (int)threadIdx.x % TPL : (int)threadIdx.x / B;   // thread within the line
    const int sign = P.sign;
    const int N = P.N, h = N / 2;

    // ---- line context
    LineIO<T> io;
    io.n = P.n;
    io.h = h;
    io.kind = P.in_kind;
    io.fac = reinterpret_cast<const T *>(P.fac);
    io.mirror_base = -1;
    io.win = P.win;
    io.bfac = T(1);
    int64_t mbase = 0;
    int xl = NF;  // ball window (modes 1, 2): |signed x index| <= xl on this row, -1: none
    LineIO<T> io2;  // packed modes: the second data column of this FFT line (set field by field)
    io2.n = P.n;
    io2.h = h;
    io2.kind = P.in_kind;
    io2.fac = io.fac;
    io2.mirror_base = -1;
    io2.win = P.win;
    io2.bfac = T(1);
    io2.valid = false;
    io2.in_base = io2.out_base = 0;
    io2.in_st = P.in_sa;
    io2.out_st = P.out_sa;
    if (!ROW) {
        constexpr int CPT = B * fft_pack(MODE);  // data columns per CTA
        const int64_t tiles = (P.I + CPT - 1) / CPT;
        const int64_t o = blockIdx.x / tiles;
        const int64_t i = (blockIdx.x % tiles) * CPT + ll;
        io.valid = i < P.I;
        io.in_base = o * P.in_so + i;
        io.out_base = o * P.out_so + i;
        io.in_st = P.in_sa;
        io.out_st = P.out_sa;
        const T *fac = reinterpret_cast<const T *>(P.fac);
        if (io.valid && (P.in_kind == IN_REAL_MODES || P.out_kind == OUT_REAL_MODES))
            io.bfac = (P.dim == 3) ? fac[i / N] * fac[i % N] : fac[i];
        if (PACK) {
            const int64_t i2 = i + B;
            io2.valid = i2 < P.I;
            io2.in_base = io.in_base + B;
            io2.out_base = io.out_base + B;
            io2.bfac = io2.valid ? ((P.dim == 3) ? fac[i2 / N] * fac[i2 % N] : fac[i2]) : T(1);
        }
        if constexpr (DUAL) {  // the same column: I_1 (io, no window) and I_2 (io2: fac2, window)
            const T *fac2 = reinterpret_cast<const T *>(P.fac2);
            io.win = 0;
            io2.fac = fac2;
            io2.valid = io.valid;
            io2.in_base = io.in_base;
            io2.out_base = io.out_base;
            io2.bfac = io2.valid ? ((P.dim == 3) ? fac2[i / N] * fac2[i % N] : fac2[i]) : T(1);
        }
    } else {
        const int64_t q = (int64_t)blockIdx.x * B + ll;
        io.valid = q < P.I;
        io.in_st = 1;
        io.out_st = 1;
        io.out_base = q * P.out_so;
        mbase = q * P.n;  // mode 5: the line's multiplier row
        // windowed 3D row pass: compact row q -> plane, full-grid row
        int64_t wz = 0, wy = 0;
        if (P.win_rows > 0) {
            wz = q / P.win_rows;
            const int64_t c = q % P.win_rows;
            wy = c <= P.win ? c : P.n - (P.win_rows - c);
            if (P.out_kind == OUT_CPLX_FULL) io.out_base = (wz * P.n + wy) * P.out_so;
        }
        if (P.in_kind == IN_CPLX_FOLD) {
            const int n = P.n;
            const int64_t lz = P.win_rows > 0 ? wz : q / P.fold_rows_per_plane;
            const int64_t ly = P.win_rows > 0 ? wy : q % P.fold_rows_per_plane;
            io.in_base = (lz + P.fold_pad) * P.fold_plane + ly * n;
            if (lz <= P.fold_pad || lz >= n / 2 - P.fold_pad) {
                const int64_t mz = (lz <= P.fold_pad) ? -lz : n - lz;
                const int64_t my = (P.fold_rows_per_plane == 1 || ly == 0) ? 0 : n - ly;
                io.mirror_base = (mz + P.fold_pad) * P.fold_plane + my * n;
            }
        } else {
            io.in_base = q * P.in_so;
        }
        if constexpr (MODE == 1 || MODE == 2 || MODE == 5) {
            if (P.ball2 > 0) {  // block-uniform branch
                const int64_t a0 = P.dim == 3 ? q / NF : q, a1 = P.dim == 3 ? q % NF : 0;
                const int64_t s1 = a1 < NF / 2 ? a1 : a1 - NF;
                const int64_t r2 = a0 * a0 + s1 * s1;
                xl = r2 > P.ball2 ? -1 : (int)sqrtf((float)(P.ball2 - r2)) + 1;
                if (MODE == 1 && xl < 0) io.valid = false;  // nothing to read or write
                if (!__syncthreads_or(io.valid && xl >= 0)) {  // every row of the CTA outside
                    if ((MODE == 2 || MODE == 5) && io.valid)  // their transforms are zero
                        for (int a = t; a < N; a += TPL)
                            reinterpret_cast<T2 *>(vout)[io.out_base + a] = czero<T2>();
                    return;
                }
            }
        }
    }
    // entry e of a row pass inside the ball window
    auto in_ball = [&](int e) { return (e <= NF / 2 ? e : NF - e) <= xl; };

    auto sidx = [&](int e) -> int { return ROW ? ll * C::ROW_LD + e + (e >> C::PADSH) : e * B + ll; };

    constexpr unsigned KM = fft_in_mask(MODE), OM = fft_out_mask(MODE);
    // ---- staged input (FP32 modes 3, 4): the CTA's 2B data columns, row by row, by cp.async
    constexpr bool STAGE = fft_stages_input(MODE, V, C::CS);
    constexpr int CPT2 = 2 * B;                                  // data columns of the CTA
    constexpr int SES = MODE == 3 ? (int)sizeof(T) : (int)sizeof(T2);  // staged element bytes
    constexpr int EPC = 16 / SES;                                // elements per 16-byte copy
    int srows = 0;
    // mode 4 with energy products also stages its density rows (N per column, floats) after the
    // input and the transform buffer; they are waited for only before the epilogue
    bool rstaged = false;
    int roff = 0;  // byte offset of the staged density
    if constexpr (STAGE && !ROW) {
        const int64_t tiles = (P.I + CPT2 - 1) / CPT2;
        const int64_t i0 = (blockIdx.x % tiles) * CPT2;
        const int64_t in0 = (blockIdx.x / tiles) * P.in_so + i0;
        {
            srows = fft_stage_rows(MODE, NF, N, P.win);
            constexpr int CPR = CPT2 / EPC;  // copies per row
            const unsigned char *src = reinterpret_cast<const unsigned char *>(vin);
            const uint32_t dst0 = (uint32_t)__cvta_generic_to_shared(smem_raw);
            for (int c = threadIdx.x; c < srows * CPR; c += blockDim.x) {
                const int row = c / CPR, k = c - row * CPR;
                if (i0 + (int64_t)k * EPC < P.I) {
                    const unsigned char *g = src + (in0 + row * P.in_sa + (int64_t)k * EPC) * SES;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst0 + (uint32_t)((row * CPT2 + k * EPC) * SES)),
                                 "l"(g)
                                 : "memory");
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            if constexpr (MODE == 4) {
                const T *rho = reinterpret_cast<const T *>(P.rho);
                constexpr int REPC = 16 / (int)sizeof(T);
                const int a = NF * B * (int)sizeof(T2), b = srows * CPT2 * SES;
                roff = ((a > b ? a : b) + 15) & ~15;
                uint32_t dsm;  // the launch's dynamic shared memory: room for the density rows?
                asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsm));
                rstaged = rho && P.I % REPC == 0 && P.out_so % REPC == 0 && P.out_sa % REPC == 0 &&
                          CPT2 % REPC == 0 && (reinterpret_cast<uintptr_t>(rho) & 15) == 0 &&
                          (uint32_t)roff + (uint32_t)(N * CPT2 * (int)sizeof(T)) <= dsm;  // uniform
                if (rstaged) {
                    const int64_t o0 = (blockIdx.x / tiles) * P.out_so + i0;
                    constexpr int RCPR = CPT2 / REPC;
                    for (int c = threadIdx.x; c < N * RCPR; c += blockDim.x) {
                        const int row = c / RCPR, k = c - row * RCPR;
                        if (i0 + (int64_t)k * REPC < P.I)
                            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                                             dst0 + (uint32_t)(roff + (row * CPT2 + k * REPC) * (int)sizeof(T))),
                                         "l"(rho + o0 + row * P.out_sa + (int64_t)k * REPC)
                                         : "memory");
                    }
                    asm volatile("cp.async.commit_group;" ::: "memory");
                }
            }
            if (rstaged) asm volatile("cp.async.wait_group 1;" ::: "memory");  // the input only
            else asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
        }
    }
    // staged entry e of data column col (0..2B-1) of the CTA, as io.load would give it
    auto sload = [&](int e, int col, const LineIO<T> &L) -> T2 {
        T2 v = czero<T2>();
        if (!L.valid) return v;
        if constexpr (MODE == 3) {
            const int m = e < NF / 2 ? e : e - NF;
            if (m >= -h && m < h) {
                const int a = m + h;
                v.x = reinterpret_cast<const T *>(smem_raw)[a * CPT2 + col] * L.fac[a] * L.bfac;
            }
        } else {
            const int f = e <= NF / 2 ? e : NF - e;
            if (f < srows) {
                v = reinterpret_cast<const T2 *>(smem_raw)[f * CPT2 + col];
                if (e > NF / 2) v = cconj(v);
            }
        }
        return v;
    };
    // ---- stage 0: global -> registers -> DFT -> shared
    int sgn = MODE == 5 ? -1 : sign;  // mode 5: forward transform first
    {
        constexpr int R = fft_radix(NF, 0, C::VG);
        constexpr int NB = NF / R;
        constexpr int MB = NB / TPL;
        T2 v[MB][R];
#pragma unroll
        for (int b = 0; b < MB; b++)
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int e = t + b * TPL + r * NB;
                if constexpr (STAGE) {  // (modes 3, 4) the two columns of this FFT line from the stage
                    if constexpr (MODE == 3) {
                        v[b][r] = cmake<T2>(sload(e, ll, io).x, sload(e, ll + B, io2).x);
                    } else {
                        const T2 X = sload(e, ll, io), Y = sload(e, ll + B, io2);
                        v[b][r] = cmake<T2>(X.x - Y.y, X.y + Y.x);
                    }
                } else if constexpr (MODE == 3 || MODE == 6) {  // z = x + i y from two real lines
                    v[b][r] = cmake<T2>(io.template load<KM>(e, vin).x, io2.template load<KM>(e, vin).x);
                } else if constexpr (MODE == 7) {  // Z = X1 + i X2, X2 from the second input
                    const T2 X = io.template load<KM>(e, vin), Y = io2.template load<KM>(e, P.in2);
                    v[b][r] = cmake<T2>(X.x - Y.y, X.y + Y.x);
                } else if constexpr (MODE == 4) {  // Z = X + i Y from two Hermitian columns
                    const T2 X = io.template load<KM>(e, vin), Y = io2.template load<KM>(e, vin);
                    v[b][r] = cmake<T2>(X.x - Y.y, X.y + Y.x);
                } else if constexpr (MODE == 2) {  // fold: the row here, the mirror row below
                    v[b][r] = (io.valid && in_ball(e)) ? reinterpret_cast<const T2 *>(vin)[io.in_base + e]
                                                       : czero<T2>();
                } else {
                    v[b][r] = io.template load<KM>(e, vin);
                }
            }
        if constexpr (MODE == 2) {  // H[l] = H+[l] + conj(H+[-l]): all mirror loads in one batch
            if (io.valid && io.mirror_base >= 0) {
                const T2 *in = reinterpret_cast<const T2 *>(vin);
                T2 m[MB][R];
#pragma unroll
                for (int b = 0; b < MB; b++)
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int e = t + b * TPL + r * NB;
                        m[b][r] = in_ball(e) ? in[io.mirror_base + (e == 0 ? 0 : NF - e)] : czero<T2>();
                    }
#pragma unroll
                for (int b = 0; b < MB; b++)
#pragma unroll
                    for (int r = 0; r < R; r++) v[b][r] = cadd(v[b][r], cconj(m[b][r]));
            }
        }
        if constexpr (STAGE) __syncthreads();  // the stage (aliasing buf) is read before buf is written
#pragma unroll
        for (int b = 0; b < MB; b++) {
            dft_small<T, R>(v[b], sgn);
            const int i = t + b * TPL;
#pragma unroll
            for (int r = 0; r < R; r++) buf[sidx(i * R + r)] = v[b][r];
        }
    }
    __syncthreads();

    // ---- stages 1 .. NST-1; the last one writes the output
    EAcc<T> eacc;  // this thread's u*rho products
    auto stage = [&](auto S_) {
        constexpr int S = decltype(S_)::value;
        constexpr int R = fft_radix(NF, S, C::VG);
        constexpr int NB = NF / R;
        constexpr int MB = NB / TPL;
        constexpr int PP = fft_pprod(NF, S, C::VG);
        constexpr int STEP = NF / (PP * R);
        constexpr bool LAST = (S == C::NST - 1);
        T2 v[MB][R];
#pragma unroll
        for (int b = 0; b < MB; b++)
#pragma unroll
            for (int r = 0; r < R; r++) v[b][r] = buf[sidx(t + b * TPL + r * NB)];
        if (!LAST || NATURAL || (MODE == 5 && sgn < 0)) __syncthreads();
#pragma unroll
        for (int b = 0; b < MB; b++) {
            const int i = t + b * TPL;
            const int k = i % PP;
#pragma unroll
            for (int r = 1; r < R; r++) {
                T2 w = tw[r * k * STEP];
                if (sgn > 0) w = cconj(w);
                v[b][r] = cmul(v[b][r], w);
            }
            dft_small<T, R>(v[b], sgn);
            if constexpr (!LAST) {
                const int j = (i - k) * R + k;
#pragma unroll
                for (int r = 0; r < R; r++) buf[sidx(j + r * PP)] = v[b][r];
            } else if constexpr (NATURAL) {  // z in natural order for the epilogue below
#pragma unroll
                for (int r = 0; r < R; r++) buf[sidx(i + r * PP)] = v[b][r];
            } else if (MODE == 5 && sgn < 0) {  // spectrum times the multiplier row, natural order
                const T *mrow = reinterpret_cast<const T *>(P.mult) + mbase;
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const int e = i + r * PP;
                    buf[sidx(e)] = cscale(v[b][r], io.valid ? mrow[e] : T(0));
                }
            } else if (io.valid) {
                // output entry e = i + r PP (here PP R = n and k = i)
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const int e = i + r * PP;
                    const T2 x = v[b][r];
                    constexpr bool OONE = (OM & (OM - 1)) == 0;
                    auto os = [&](int k) { return (OM & (1u << k)) != 0 && (OONE || P.out_kind == k); };
                    if (os(OUT_CPLX_FULL)) {
                        if ((P.win == 0 || e <= P.win || e >= NF - P.win) && (MODE != 1 || in_ball(e)))
                            reinterpret_cast<T2 *>(vout)[io.out_base + e * io.out_st] = x;
                    } else if (os(OUT_CPLX_HALF)) {
                        if (e <= (P.win > 0 ? P.win : NF / 2))
                            reinterpret_cast<T2 *>(vout)[io.out_base + e * io.out_st] = x;
                    } else if (os(OUT_CPLX_WIN)) {
                        const int c = e <= P.win ? e : (e >= NF - P.win ? e - NF + 2 * P.win + 1 : -1);
                        if (c >= 0) reinterpret_cast<T2 *>(vout)[io.out_base + c * io.out_st] = x;
                    } else if (os(OUT_CPLX_MODES)) {
                        const int m = e < NF / 2 ? e : e - NF;
                        if (m >= -h && m < h)
                            reinterpret_cast<T2 *>(vout)[io.out_base + (m + h) * io.out_st] = x;
                    } else if (os(OUT_REAL_MODES)) {  // (+ energy)
                        const int m = e < NF / 2 ? e : e - NF;
                        if (m >= -h && m < h) {
                            const int a = m + h;
                            const T *fac = reinterpret_cast<const T *>(P.fac);
                            const int64_t idx = io.out_base + a * io.out_st;
                            T val = x.x * fac[a] * io.bfac;
                            if (P.accum) val += reinterpret_cast<const T *>(vout)[idx];
                            reinterpret_cast<T *>(vout)[idx] = val;
                            if (P.rho) eacc.add(val, reinterpret_cast<const T *>(P.rho)[idx]);
                        }
                    }
                }
            }
        }
        if constexpr (!LAST) __syncthreads();
    };
    static_for<1, C::NST>(stage);
    if constexpr (MODE == 5) {  // the inverse transform of the multiplied line (natural order)
        __syncthreads();
        sgn = +1;
        constexpr int R = fft_radix(NF, 0, C::VG);
        constexpr int NB = NF / R;
        constexpr int MB = NB / TPL;
        T2 v[MB][R];
#pragma unroll
        for (int b = 0; b < MB; b++)
#pragma unroll
            for (int r = 0; r < R; r++) v[b][r] = buf[sidx(t + b * TPL + r * NB)];
        __syncthreads();  // every input read before buf is rewritten
#pragma unroll
        for (int b = 0; b < MB; b++) {
            dft_small<T, R>(v[b], sgn);
            const int i = t + b * TPL;
#pragma unroll
            for (int r = 0; r < R; r++) buf[sidx(i * R + r)] = v[b][r];
        }
        __syncthreads();
        static_for<1, C::NST>(stage);
    }

    if constexpr (MODE == 4) {  // x = Re z, y = Im z at the stored modes (+ energy)
        if (rstaged) asm volatile("cp.async.wait_group 0;" ::: "memory");  // the staged density
        __syncthreads();
        const T *fac = reinterpret_cast<const T *>(P.fac);
        const T *rho = reinterpret_cast<const T *>(P.rho);
        const T *rs = reinterpret_cast<const T *>(smem_raw + roff);
#pragma unroll 4
        for (int a = t; a < N; a += TPL) {
            const int m = a - h;
            const T2 z = buf[sidx(m < 0 ? m + NF : m)];
            const T f = fac[a];
            if (io.valid) {
                const int64_t idx = io.out_base + a * io.out_st;
                T val = z.x * f * io.bfac;
                if (P.accum) val += reinterpret_cast<const T *>(vout)[idx];
                reinterpret_cast<T *>(vout)[idx] = val;
                if (rho) eacc.add(val, rstaged ? rs[a * (2 * B) + ll] : rho[idx]);
            }
            if (io2.valid) {
                const int64_t idx = io2.out_base + a * io2.out_st;
                T val = z.y * f * io2.bfac;
                if (P.accum) val += reinterpret_cast<const T *>(vout)[idx];
                reinterpret_cast<T *>(vout)[idx] = val;
                if (rho) eacc.add(val, rstaged ? rs[a * (2 * B) + ll + B] : rho[idx]);
            }
        }
    }
    if constexpr (MODE == 7) {  // u = Re z (I_1, unit factors) + Im z times I_2's deconvolution
        __syncthreads();
        const T *fac2 = reinterpret_cast<const T *>(P.fac2);
        const T *rho = reinterpret_cast<const T *>(P.rho);
#pragma unroll 4
        for (int a = t; a < N; a += TPL) {
            const int m = a - h;
            const T2 z = buf[sidx(m < 0 ? m + NF : m)];
            if (io.valid) {
                const int64_t idx = io.out_base + a * io.out_st;
                const T val = z.x + z.y * fac2[a] * io2.bfac;
                reinterpret_cast<T *>(vout)[idx] = val;
                if (rho) eacc.add(val, rho[idx]);
            }
        }
    }
    if constexpr (MODE == 6) {  // X1 (half) to the output, X2 (window) to out2
        __syncthreads();
        for (int k = t; k <= NF / 2; k += TPL) {
            const T2 zk = buf[sidx(k)], zn = buf[sidx(k == 0 ? 0 : NF - k)];
            if (io.valid) {
                reinterpret_cast<T2 *>(vout)[io.out_base + k * io.out_st] =
                    cmake<T2>(T(0.5) * (zk.x + zn.x), T(0.5) * (zk.y - zn.y));
                if (k <= P.win)
                    reinterpret_cast<T2 *>(P.out2)[io.out_base + k * io.out_st] =
                        cmake<T2>(T(0.5) * (zk.y + zn.y), T(0.5) * (zn.x - zk.x));
            }
        }
    }
    if constexpr (MODE == 3) {  // X(k) = (Z(k) + conj Z(n-k)) / 2, Y(k) = (Z(k) - conj Z(n-k)) / 2i
        __syncthreads();
        const int klim = P.win > 0 ? P.win : NF / 2;  // OUT_CPLX_HALF (within the window)
        for (int k = t; k <= klim; k += TPL) {
            const T2 zk = buf[sidx(k)], zn = buf[sidx(k == 0 ? 0 : NF - k)];
            if (io.valid)
                reinterpret_cast<T2 *>(vout)[io.out_base + k * io.out_st] =
                    cmake<T2>(T(0.5) * (zk.x + zn.x), T(0.5) * (zk.y - zn.y));
            if (io2.valid)
                reinterpret_cast<T2 *>(vout)[io2.out_base + k * io2.out_st] =
                    cmake<T2>(T(0.5) * (zk.y + zn.y), T(0.5) * (zn.x - zk.x));
        }
    }

    if (P.out_kind == OUT_REAL_MODES && P.partials) {  // (modes 4, 7 and the column passes)
        __syncthreads();  // the shared buffer becomes the reduction scratch
        const double2 tot = energy_block_sum(eacc, reinterpret_cast<double *>(smem_raw));
        if (threadIdx.x == 0) P.partials[blockIdx.x] = tot;
    }
}

// ------------------------------------------------------------------ launchers
// kernel variant 2 applies: FP32 packed pass of schedule 0 whose staged rows are 16-byte runs
template <typename T, int MODE>
bool fft_stage_ok(const PassDesc &p, const void *in) {
    if (!fft_stages_input(MODE, 2, (int)(2 * sizeof(T))) || p.sched != 0) return false;
    const int64_t epc = 16 / (MODE == 3 ? (int64_t)sizeof(T) : (int64_t)(2 * sizeof(T)));
    return (2 * p.B) % epc == 0 && p.I % epc == 0 && p.in_so % epc == 0 && p.in_sa % epc == 0 &&
           (reinterpret_cast<uintptr_t>(in) & 15) == 0;
}

template <typename T, int NF, int MODE, int V>
cudaError_t launch_nf(const PassDesc &p, const void *in, void *out, const void *tw, cudaStream_t s) {
    if (!(fft_in_mask(MODE) & (1u << p.in_kind)) || !(fft_out_mask(MODE) & (1u << p.out_kind)))
        return cudaErrorInvalidValue;  // a pass descriptor this mode was not compiled for
    if (fft_dual(MODE) && (!p.fac2 || (MODE == 6 ? !p.out2 : !p.in2) || p.win <= 0 || p.win > NF / 2))
        return cudaErrorInvalidValue;  // a dual pass needs its second factors, buffer and window
    if (p.TPC != FftCfg<T, NF, MODE, V>::TPL || p.B != FftCfg<T, NF, MODE, V>::B ||
        (fft_is_row(MODE) && p.LD != FftCfg<T, NF, MODE, V>::ROW_LD))
        return cudaErrorInvalidValue;  // the descriptor was configured for another schedule
    const size_t smem = pass_smem(p, sizeof(T) == 4 ? NLINT_FP32 : NLINT_FP64);
    cudaError_t e = cudaFuncSetAttribute(fft_pass_kernel<T, NF, MODE, V>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t nb = pass_blocks(p, fft_is_row(MODE));
    if (nb == 0) return cudaSuccess;
    e = launch_pdl(fft_pass_kernel<T, NF, MODE, V>, dim3((unsigned)nb), dim3(FftCfg<T, NF, MODE, V>::THREADS),
                   smem, s, p, in, out, reinterpret_cast<const cx_t<T> *>(tw));
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Schedule V of every supported length; for V = 1 a length without a second schedule runs
// schedule 0 (launch_pass_mode_v<T, MODE, 0>, instantiated in its own translation unit).
template <typename T, int NF, int MODE, int V>
cudaError_t launch_nf_v(const PassDesc &p, const void *in, void *out, const void *tw, cudaStream_t s) {
    if constexpr (V == 1 && !fft_has_alt(NF, MODE)) return launch_pass_mode_v<T, MODE, 0>(p, in, out, tw, s);
    else if constexpr (V == 2 && !fft_stages_input(MODE, 2, (int)(2 * sizeof(T))))
        return launch_pass_mode_v<T, MODE, 0>(p, in, out, tw, s);
    else return launch_nf<T, NF, MODE, V>(p, in, out, tw, s);
}

template <typename T, int MODE, int V>
cudaError_t launch_pass_mode_v(const PassDesc &p, const void *in, void *out, const void *tw, cudaStream_t s) {
    switch (p.n) {
        case 16: return launch_nf_v<T, 16, MODE, V>(p, in, out, tw, s);
        case 24: return launch_nf_v<T, 24, MODE, V>(p, in, out, tw, s);
        case 32: return launch_nf_v<T, 32, MODE, V>(p, in, out, tw, s);
        case 48: return launch_nf_v<T, 48, MODE, V>(p, in, out, tw, s);
        case 64: return launch_nf_v<T, 64, MODE, V>(p, in, out, tw, s);
        case 96: return launch_nf_v<T, 96, MODE, V>(p, in, out, tw, s);
        case 128: return launch_nf_v<T, 128, MODE, V>(p, in, out, tw, s);
        case 192: return launch_nf_v<T, 192, MODE, V>(p, in, out, tw, s);
        case 256: return launch_nf_v<T, 256, MODE, V>(p, in, out, tw, s);
        case 384: return launch_nf_v<T, 384, MODE, V>(p, in, out, tw, s);
        case 512: return launch_nf_v<T, 512, MODE, V>(p, in, out, tw, s);
        case 768: return launch_nf_v<T, 768, MODE, V>(p, in, out, tw, s);
        case 1024: return launch_nf_v<T, 1024, MODE, V>(p, in, out, tw, s);
        case 1536: return launch_nf_v<T, 1536, MODE, V>(p, in, out, tw, s);
        case 2048: return launch_nf_v<T, 2048, MODE, V>(p, in, out, tw, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace nlint
