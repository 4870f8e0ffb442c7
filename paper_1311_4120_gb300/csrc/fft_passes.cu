// Host side of the oversampled-grid FFT passes: supported sizes, CTA geometry and dispatch to
// the per-(precision, direction) translation units that hold the kernels (fft_kernels.cuh).
#include "fft_kernels.cuh"

namespace nlint {

// the kernels are instantiated in fft_{f32,f64}_{col,row,rowr,colp,conv,dual}.cu (schedule 0) and
// fft_f32_{col,row,rowr,colp}_s1.cu (schedule 1) and fft_f32_colp_s2.cu (staged input)
extern template cudaError_t launch_pass_mode_v<float, 0, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 1, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 2, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 3, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 4, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 5, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 6, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 7, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<double, 0, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<double, 1, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<double, 2, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<double, 3, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<double, 4, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<double, 5, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<double, 6, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<double, 7, 0>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 0, 1>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 1, 1>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 2, 1>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 3, 1>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 4, 1>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 3, 2>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
extern template cudaError_t launch_pass_mode_v<float, 4, 2>(const PassDesc &, const void *, void *, const void *, cudaStream_t);

int pass_mode(const PassDesc &p, bool row) {
    if (!row) {
        if (p.dual) return p.in_kind == IN_REAL_MODES ? 6 : 7;
        if (p.in_kind == IN_REAL_MODES && p.out_kind == OUT_CPLX_HALF) return 3;
        if (p.in_kind == IN_CPLX_HERM && p.out_kind == OUT_REAL_MODES) return 4;
        return 0;
    }
    if (p.conv) return 5;
    return p.in_kind == IN_CPLX_FOLD ? 2 : 1;
}

bool fft_size_supported(int n) {
    if (n < 16 || n > 2048) return false;
    const int m = (n % 3 == 0) ? n / 3 : n;
    return m >= 8 && (m & (m - 1)) == 0;
}

int fft_next_size(int64_t m) {
    static const int sizes[] = {16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048};
    for (int s : sizes)
        if (s >= m) return s;
    return -1;
}

void make_radix(int n, PassDesc &p) {
    p.nrad = 0;
    if (!fft_size_supported(n)) {
        p.nrad = -1;
        return;
    }
    int m = n % 3 == 0 ? n / 3 : n, k = 0;
    while (m % 8 == 0) {
        p.rad[k++] = 8;
        m /= 8;
    }
    if (m == 4) p.rad[k++] = 4;
    if (m == 2) p.rad[k++] = 2;
    if (n % 3 == 0) p.rad[k++] = 3;
    p.nrad = k;
}

void config_pass(PassDesc &p, int prec, bool row, unsigned sched) {
    const int cs = prec == NLINT_FP32 ? 8 : 16;
    const int mode = pass_mode(p, row);
    const int bit = mode == 0 ? 0 : mode == 1 ? 1 : mode == 2 ? 2 : (mode == 3 || mode == 4) ? 3 : -1;
    p.sched = (prec == NLINT_FP32 && bit >= 0 && fft_has_alt(p.n, mode)) ? (int)((sched >> bit) & 1u) : 0;
    p.TPC = fft_tpl(p.n, mode, p.sched);
    p.B = row ? fft_row_b(p.n, cs, mode, p.sched) : fft_col_b_m(p.n, cs, mode, p.sched);
    p.LD = row ? fft_row_ld(p.n, p.sched) : p.B;
}

template <typename T, int MODE>
cudaError_t launch_pass_mode(const PassDesc &p, const void *in, void *out, const void *tw, cudaStream_t s) {
    if constexpr (sizeof(T) == 4 && MODE <= 4)
        if (p.sched) return launch_pass_mode_v<T, MODE, 1>(p, in, out, tw, s);
    if constexpr (sizeof(T) == 4 && (MODE == 3 || MODE == 4))
        if (fft_stage_ok<T, MODE>(p, in)) return launch_pass_mode_v<T, MODE, 2>(p, in, out, tw, s);
    return launch_pass_mode_v<T, MODE, 0>(p, in, out, tw, s);
}

int pass_threads(const PassDesc &p) { return p.B * p.TPC; }

bool pass_fits(const PassDesc &p) { return p.nrad > 0 && pass_threads(p) <= 1024; }

int64_t pass_blocks(const PassDesc &p, bool row) {
    if (row) return (p.I + p.B - 1) / p.B;
    const int cpt = p.B * fft_pack(pass_mode(p, false));  // data columns per CTA
    return p.n_outer * ((p.I + cpt - 1) / cpt);
}

size_t pass_smem(const PassDesc &p, int prec) {
    const size_t cs = (prec == NLINT_FP32) ? 8 : 16;
    const size_t a = (size_t)p.B * p.LD * cs, b = (size_t)p.n * p.B * cs;
    size_t s = a > b ? a : b;
    const int mode = pass_mode(p, false);
    if (fft_stages_input(mode, p.sched == 0 ? 2 : 1, (int)cs)) {  // variant 2's staged input rows
        const size_t es = mode == 3 ? cs / 2 : cs;
        const size_t st = (size_t)fft_stage_rows(mode, p.n, p.N, p.win) * 2 * p.B * es;
        if (st > s) s = st;
        // + the density rows of mode 4 when they fit (the kernel checks its shared memory)
        const size_t with_rho = ((s + 15) & ~(size_t)15) + (size_t)p.N * 2 * p.B * (cs / 2);
        if (mode == 4 && with_rho <= 200 * 1024) s = with_rho;
    }
    return s > 64 * sizeof(double) ? s : 64 * sizeof(double);  // >= the energy scratch
}

template <typename T>
cudaError_t launch_colpass(const PassDesc &p, const void *in, void *out, const void *tw, cudaStream_t s) {
    switch (pass_mode(p, false)) {
        case 3: return launch_pass_mode<T, 3>(p, in, out, tw, s);
        case 4: return launch_pass_mode<T, 4>(p, in, out, tw, s);
        case 6: return launch_pass_mode<T, 6>(p, in, out, tw, s);
        case 7: return launch_pass_mode<T, 7>(p, in, out, tw, s);
        default: return launch_pass_mode<T, 0>(p, in, out, tw, s);
    }
}

template <typename T>
cudaError_t launch_rowpass(const PassDesc &p, const void *in, void *out, const void *tw, cudaStream_t s) {
    switch (pass_mode(p, true)) {
        case 2: return launch_pass_mode<T, 2>(p, in, out, tw, s);
        case 5: return launch_pass_mode<T, 5>(p, in, out, tw, s);
        default: return launch_pass_mode<T, 1>(p, in, out, tw, s);
    }
}

template cudaError_t launch_colpass<float>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
template cudaError_t launch_colpass<double>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
template cudaError_t launch_rowpass<float>(const PassDesc &, const void *, void *, const void *, cudaStream_t);
template cudaError_t launch_rowpass<double>(const PassDesc &, const void *, void *, const void *, cudaStream_t);

}  // namespace nlint
