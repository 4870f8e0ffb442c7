// Shared device helpers: complex arithmetic on float2/double2 and precision traits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nlint {

template <typename T> struct Cx;
template <> struct Cx<float> { using T2 = float2; };
template <> struct Cx<double> { using T2 = double2; };
template <typename T> using cx_t = typename Cx<T>::T2;

template <typename T2> __device__ __forceinline__ T2 cmake(decltype(T2{}.x) a, decltype(T2{}.x) b) {
    T2 r; r.x = a; r.y = b; return r;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// multiply by sign*i: (x + iy) * (s i) = -s y + i s x
__device__ __forceinline__ float2 cmuli(float2 a, int s) { return make_float2(-s * a.y, s * a.x); }
__device__ __forceinline__ double2 cmuli(double2 a, int s) { return make_double2(-s * a.y, s * a.x); }
template <typename T2> __device__ __forceinline__ T2 czero() { T2 r; r.x = 0; r.y = 0; return r; }

// Programmatic dependent launch.  A kernel launched by launch_pdl may be scheduled while the
// kernel before it on the stream is still finishing: it calls pdl_wait() first, which returns
// once that kernel has completed and its writes are visible (so it reads and writes nothing
// earlier), then pdl_trigger(), which lets the kernel after it be scheduled in turn.  Only the
// launch latency and the CTA scheduling overlap; the stream order of the data is unchanged.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Compile-time loop: f(IntC<B>{}), f(IntC<B+1>{}), ..., f(IntC<E-1>{}).
template <int V> struct IntC { static constexpr int value = V; };
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (B < E) {
        f(IntC<B>{});
        static_for<B + 1, E>(f);
    }
}

// Neumaier-compensated FP64 accumulator: s + c carries the sum.
struct KSum {
    double s, c;
    __device__ __forceinline__ void init() { s = 0.0; c = 0.0; }
    __device__ __forceinline__ void add(double x) {
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return s + c; }
    // absorb another compensated sum (its value s + c)
    __device__ __forceinline__ void merge(double os, double oc) { add(os); add(oc); }
};

// Deterministic reduction of a compensated sum over a warp: a fixed butterfly of shuffles,
// so the result depends only on the lane values, never on timing.
__device__ __forceinline__ void ksum_warp(KSum &k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double os = __shfl_down_sync(0xffffffffu, k.s, off);
        const double oc = __shfl_down_sync(0xffffffffu, k.c, off);
        k.merge(os, oc);
    }
}

// Deterministic CTA reduction (blockDim.x a multiple of 32, <= 1024); the total is valid in
// thread 0.  `scratch` holds 2 doubles per warp.
__device__ __forceinline__ KSum ksum_block(KSum k, double *scratch) {
    ksum_warp(k);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        scratch[2 * wid] = k.s;
        scratch[2 * wid + 1] = k.c;
    }
    __syncthreads();
    KSum t;
    t.init();
    if (wid == 0) {
        if (lane < nw) {
            t.s = scratch[2 * lane];
            t.c = scratch[2 * lane + 1];
        }
        ksum_warp(t);
    }
    return t;
}

// Energy accumulator of one thread: sum of u*rho products.  FP32 inputs: the exact product
// p + e (p = u*rho rounded, e = fma(u, rho, -p)) is summed in FP32 with Kahan compensation, so
// no FP64 instruction runs per grid point (FP64 throughput is a small fraction of FP32 on this
// GPU); FP64 inputs: FP64 FMA into a running sum.
template <typename T> struct EAcc;
template <> struct EAcc<float> {
    float s = 0.f, c = 0.f, e = 0.f;
    __device__ __forceinline__ void add(float u, float r) {
        const float p = u * r;
        e += fmaf(u, r, -p);
        const float y = p - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    // (hi, lo) with hi + lo the compensated sum
    __device__ __forceinline__ float hi() const { return s; }
    __device__ __forceinline__ float lo() const { return e - c; }
};
template <> struct EAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double u, double r) { s = fma(u, r, s); }
};

// Float-float addition (TwoSum): (a_hi + a_lo) + (b_hi + b_lo) to about 2^-44 relative.
__device__ __forceinline__ void ff_add(float &hi, float &lo, float bhi, float blo) {
    const float s = hi + bhi;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (bhi - bb);
    const float l = lo + blo + err;
    hi = s + l;
    lo = l - (hi - s);
}

// CTA sum of the threads' energy accumulators into one compensated FP64 partial (valid in
// thread 0).  FP32: a float-float shuffle tree per warp, then one warp folds the warp sums in
// FP64; FP64: the compensated FP64 tree.  The order is fixed, so results are reproducible.
// `scratch` holds 2 doubles per warp; blockDim.x must be a multiple of 32.
__device__ __forceinline__ double2 energy_block_sum(const EAcc<float> &a, double *scratch) {
    float hi = a.hi(), lo = a.lo();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ohi = __shfl_down_sync(0xffffffffu, hi, off);
        const float olo = __shfl_down_sync(0xffffffffu, lo, off);
        ff_add(hi, lo, ohi, olo);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        scratch[2 * wid] = (double)hi;
        scratch[2 * wid + 1] = (double)lo;
    }
    __syncthreads();
    KSum t;
    t.init();
    if (wid == 0) {
        if (lane < nw) t.merge(scratch[2 * lane], scratch[2 * lane + 1]);
        ksum_warp(t);
    }
    return make_double2(t.s, t.c);
}
__device__ __forceinline__ double2 energy_block_sum(const EAcc<double> &a, double *scratch) {
    KSum k;
    k.init();
    k.add(a.s);
    KSum t = ksum_block(k, scratch);
    return make_double2(t.s, t.c);
}

}  // namespace nlint
