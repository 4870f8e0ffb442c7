// Type-2 interpolation with the multiply by W_j, and type-1 spreading (steps a3, a4 and a5 of
// the path; Algorithm 1, eq. 3.2 and eq. 3.7), templated on the stencil width so that every
// loop over the stencil is unrolled and every tile index is a compile-time product.
//
// Spreading function: the "exponential of semicircle" of Barnett, Magland and af Klinteberg
// (SIAM J. Sci. Comput. 2019), phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1, with
// z = (l - g) / (w/2) for fine cell l and node position g in fine-cell units.  The nodes are
// fixed per plan, so the plan evaluates phi for every node and axis once, in FP64.
//
// Only the half node set (k on the non-negative side of array axis 0) is processed:
// rho_hat(-k) = conj(rho_hat(k)) for a real density, and the mirrored nodes' spreading is
// restored by the fold in the first inverse FFT pass.  The fine grid G holds the planes
// 0..n/2 of axis 0; other planes are read as conj(G[-l]).  The spread grid H+ is stored on
// planes -pad..n/2+pad of axis 0.
//
// Work decomposition: one CTA per subproblem (a run of nodes of one bin).  The CTA stages its
// bin's tile (bin + w - 1 cells per axis) in shared memory as separate real and imaginary
// planes.  Each warp owns a contiguous run of the subproblem's nodes and takes one (32 lanes
// per node) or two (16 lanes per node, when w*w fills 16-lane passes better) at a time; in 3D
// a node's lanes own (axis 1, axis 2) stencil columns and run along axis 0 with the axis-0
// kernel values in registers, in 2D they own stencil cells.
// The columns are dealt to lanes by a plan-made table so that a pass hits distinct shared-
// memory banks.  Interpolation sums the lanes with a shuffle tree; spreading adds into the
// tile with shared integer atomics (fixed point, see FixAcc; the lanes of one node touch
// distinct cells) and then adds the tile's nonzero cells to H+ with global atomics, or, for
// crowded bins, to an FP64 tile.
#pragma once
#include "common.cuh"
#include "internal.h"

#include <climits>

namespace nlint {

static constexpr int MAXW = NODE_MAXW;
static constexpr int SUB_THREADS = NODE_THREADS;

template <typename T, int D, int W>
struct Geo {
    static constexpr bool F64 = sizeof(T) == 8;
    static constexpr int B0 = bin_extent(F64, D, W, 0), B1 = bin_extent(F64, D, W, 1);
    static constexpr int B2 = (D == 3) ? bin_extent(F64, D, W, 2) : 1;
    static constexpr int T0 = B0 + W - 1, T1 = B1 + W - 1, T2 = (D == 3) ? B2 + W - 1 : 1;
    static constexpr int NCELL = T0 * T1 * T2;
    static constexpr int PAIRS = W * W;  // stencil columns per node
    // lanes per node: 16 (two nodes per warp) when that wastes fewer lane slots, else 32
    static constexpr int LPN = node_lanes(W);
    static constexpr int NPW = 32 / LPN;                 // nodes per warp iteration
    static constexpr int PASSES = (PAIRS + LPN - 1) / LPN;
};

// l mod n for l in [-n, 2n)
__device__ __forceinline__ int wrap1(int l, int n) { return l < 0 ? l + n : (l >= n ? l - n : l); }

__device__ __forceinline__ int wrapn(int l, int n) {
    int r = l % n;
    return r < 0 ? r + n : r;
}

// G at (l0, l1[, l2]) of the full periodic fine grid from its stored half (planes 0..n/2 of
// axis 0), using G[-l] = conj(G[l]) for the other half.
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

// A warp works on NPW = 32 / LPN nodes at a time (one per LPN-lane group): per node its lanes
// share the w*w stencil columns, and the nodes share the warp's per-node work (loads, shuffle
// reductions).  NodeGroup holds this lane's view: the stencil origin of its group's node
// (relative to the bin) and its share of the group's NPW*D*w kernel values, which the plan
// computed once (the nodes are fixed).
template <typename T, int D, int W>
struct NodeGroup {
    static constexpr int LPN = Geo<T, D, W>::LPN, NPW = Geo<T, D, W>::NPW;
    static constexpr int NKV = NPW * D * W;        // kernel values of the group
    static constexpr int KV = (NKV + 31) / 32;     // ... per lane
    int r0, r1, r2;
    T kv[KV];
    // nodes j .. j + NPW - 1 of the chunk ending at jb, node j + lane / LPN for this lane
    __device__ __forceinline__ void load(const NodeDesc &nd, int j, int jb, int lane) {
        const int mine = (NPW == 1) ? j : j + lane / LPN;
        const int rl = (NPW == 1 || mine < jb) ? nd.rel[mine] : 0;
        r0 = rl & 255;
        r1 = (rl >> 8) & 255;
        r2 = (rl >> 16) & 255;
        const T *ker = reinterpret_cast<const T *>(nd.ker) + (int64_t)j * (D * W);
        const int navail = (jb - j) * (D * W);  // kernel values left in the chunk
#pragma unroll
        for (int v = 0; v < KV; v++) {
            const int t = lane + 32 * v;
            kv[v] = (t < NKV && t < navail) ? ker[t] : T(0);
        }
    }
};

// Slot of this lane's v-th kernel value in the warp's table ker[h*3*MAXW + a*MAXW + q] (node h
// of the group, stencil cell q of axis a), or -1; depends on the lane only, so it is computed
// once per thread.
template <typename T, int D, int W>
__device__ __forceinline__ int kernel_slot(int lane, int v) {
    const int t = lane + 32 * v;
    if (t >= NodeGroup<T, D, W>::NKV) return -1;
    const int h = (NodeGroup<T, D, W>::NPW == 1) ? 0 : t / (D * W);
    const int rem = t - h * D * W, a = rem / W, q = rem - a * W;
    return h * 3 * MAXW + a * MAXW + q;
}

// Kernel values of the group into the warp's table.
template <typename T, int D, int W>
__device__ __forceinline__ void warp_kernel_values(const NodeGroup<T, D, W> &np, const int *slot, T *ker) {
#pragma unroll
    for (int v = 0; v < NodeGroup<T, D, W>::KV; v++)
        if (slot[v] >= 0) ker[slot[v]] = np.kv[v];
}

// Decompose a tile cell into its per-axis offsets.
template <typename G_>
__device__ __forceinline__ void cell_coords(int cell, int &a0, int &a1, int &a2) {
    a0 = cell / (G_::T1 * G_::T2);
    const int rem = cell - a0 * (G_::T1 * G_::T2);
    a1 = rem / G_::T2;
    a2 = rem - a1 * G_::T2;
}

// Tile offset of stencil column (qa, qb) for the origin (r0, r1, r2), axis-0 run start:
// origin_index(r0, r1, r2) + column_offset(qa, qb).
template <typename G_, int D>
__device__ __forceinline__ int origin_index(int r0, int r1, int r2) {
    return (D == 3) ? (r0 * G_::T1 + r1) * G_::T2 + r2 : r0 * G_::T1 + r1;
}
template <typename G_, int D>
__device__ __forceinline__ int column_offset(int qa, int qb) {
    return (D == 3) ? qa * G_::T2 + qb : qa * G_::T1 + qb;
}

// Each warp owns a contiguous run of its subproblem's nodes.
// (32-bit: a subproblem holds at most 2^20 nodes; the warp count is the compile-time
// SUB_THREADS / 32, so the division is a shift.)
__device__ __forceinline__ void warp_chunk(int4 sb, int wid, int &ja, int &jb) {
    constexpr int NW = SUB_THREADS / 32;
    ja = sb.x + (sb.y * wid) / NW;
    jb = sb.x + (sb.y * (wid + 1)) / NW;
}

// Fixed-point accumulation of the spreading tile.  Shared-memory floating-point atomics are
// several times slower than integer ones on this GPU, so each CTA adds integer multiples of
// 1/S: S = 2^(E - ceil(log2 B)) with B >= max(sum_j |Re c_j|, sum_j |Im c_j|) over the
// subproblem (every cell sum and every contribution is at most B, since phi <= 1), E = 29 for
// FP32 (int32 cells) and 50 for FP64 (int64 cells), so no cell can overflow.  Each
// contribution a * b is rounded to 1/S <= 2^-E B (FP32: 2^-29 B, finer than FP32 rounding of the
// largest cells; FP64: 2^-50 B); the integer sums are exact, so a tile does not depend on the
// order of its additions.  FP64 rounds with one fused multiply-add: a * b + 1.5 * 2^52 lies in
// [2^52, 2^53) for |a * b| < 2^51, where the spacing of doubles is 1, so its low mantissa bits
// are a * b rounded to the nearest integer (the classic magic-number conversion) -- one
// operation on the FP64 units, which bound the FP64 path, instead of a multiply and a convert.
template <typename T> struct FixAcc;
template <> struct FixAcc<float> {
    using A = int;
    static constexpr int E = 29, MAXEXP = 126;
    __device__ __forceinline__ static A mulq(float a, float b) { return __float2int_rn(a * b); }
    __device__ __forceinline__ static void add(A *p, A v) { atomicAdd(p, v); }
};
template <> struct FixAcc<double> {
    using A = long long;
    static constexpr int E = 50, MAXEXP = 1000;
    __device__ __forceinline__ static A mulq(double a, double b) {
        constexpr double MAGIC = 6755399441055744.0;  // 1.5 * 2^52
        return __double_as_longlong(fma(a, b, MAGIC)) - __double_as_longlong(MAGIC);
    }
    __device__ __forceinline__ static void add(A *p, A v) {
        atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
    }
};

template <typename T, int D, int W, bool EN>
__global__ void __launch_bounds__(SUB_THREADS) interp_sub_kernel(NodeDesc nd,
                                                                const cx_t<T> *__restrict__ G,
                                                                cx_t<T> *__restrict__ c_out,
                                                                int apply_W,
                                                                double2 *__restrict__ epart) {
    using T2 = cx_t<T>;
    using G_ = Geo<T, D, W>;
    constexpr int PASSES = G_::PASSES, L = (D == 3) ? W : 1, PLANE = G_::T1 * G_::T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the tile as real and imaginary planes (measured faster than interleaved complex, whose
    // one 8-byte load per stencil cell cost registers and resident CTAs)
    T *tr = reinterpret_cast<T *>(smem_raw);
    T *ti = tr + G_::NCELL;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int nw = SUB_THREADS / 32;  // the kernels are launched with SUB_THREADS threads
    T *ker = ti + G_::NCELL + wid * 6 * MAXW;
    const int4 sb = nd.subs[blockIdx.x];
    const int4 bo = nd.bins[sb.z];
    const int n = nd.n;
    // this lane's stencil columns, one per pass (-1: idle), as tile offsets and kernel-table
    // offsets of the two column axes; its slots in the warp's kernel table
    int coff[PASSES], kab_off[PASSES], kslot[NodeGroup<T, D, W>::KV];
#pragma unroll
    for (int ps = 0; ps < PASSES; ps++) {
        const int pq = nd.pair_order_i[ps * G_::LPN + lane % G_::LPN];
        const int qa = pq >> 8, qb = pq & 255;
        coff[ps] = pq >= 0 ? column_offset<G_, D>(qa, qb) : -1;
        kab_off[ps] = (D == 3) ? (MAXW + qa) | ((2 * MAXW + qb) << 16) : qa | ((MAXW + qb) << 16);
    }
#pragma unroll
    for (int v = 0; v < NodeGroup<T, D, W>::KV; v++) kslot[v] = kernel_slot<T, D, W>(lane, v);

    // stage the tile; the common case (axis-0 planes inside the stored half) needs no mirror
    const bool inside = bo.x >= 0 && bo.x + G_::T0 - 1 <= n / 2;
    if (D == 3 && inside) {
        // by (axis-1, axis-2) column: its wrapped offsets and base index once, then the T0
        // planes at a constant stride (no per-cell index decomposition)
        const int64_t nn = (int64_t)n * n;
        for (int col = threadIdx.x; col < PLANE; col += blockDim.x) {
            const int a1 = col / G_::T2, a2 = col - a1 * G_::T2;
            const T2 *g = G + ((int64_t)bo.x * n + wrap1(bo.y + a1, n)) * n + wrap1(bo.z + a2, n);
            constexpr int GRP = 4;  // planes in flight per thread (bounds the registers)
#pragma unroll 1
            for (int a0b = 0; a0b < G_::T0; a0b += GRP) {
                T2 v[GRP];
#pragma unroll
                for (int k = 0; k < GRP; k++)
                    if (a0b + k < G_::T0) v[k] = g[(a0b + k) * nn];
#pragma unroll
                for (int k = 0; k < GRP; k++)
                    if (a0b + k < G_::T0) {
                        tr[(a0b + k) * PLANE + col] = v[k].x;
                        ti[(a0b + k) * PLANE + col] = v[k].y;
                    }
            }
        }
    } else {
        for (int cell = threadIdx.x; cell < G_::NCELL; cell += blockDim.x) {
            int a0, a1, a2;
            cell_coords<G_>(cell, a0, a1, a2);
            T2 v;
            if (inside) {
                const int l0 = bo.x + a0, l1 = wrap1(bo.y + a1, n);
                v = (D == 3) ? G[((int64_t)l0 * n + l1) * n + wrap1(bo.z + a2, n)] : G[(int64_t)l0 * n + l1];
            } else {
                v = fetch_half<T, D>(G, n, bo.x + a0, bo.y + a1, bo.z + a2);
            }
            tr[cell] = v.x;
            ti[cell] = v.y;
        }
    }
    __syncthreads();

    int ja, jb;
    warp_chunk(sb, wid, ja, jb);
    const int half = lane / G_::LPN, hl = lane % G_::LPN;  // node of the group, lane in it
    const T *kh = ker + half * 3 * MAXW;  // this lane's node's kernel values
    NodeGroup<T, D, W> cur, nxt;
    EAcc<T> eacc;  // energy-only mode: sum of W_j |rho_hat_j|^2 over this lane's nodes
    if (ja < jb) cur.load(nd, ja, jb, lane);
    for (int j = ja; j < jb; j += G_::NPW) {
        if (j + G_::NPW < jb) nxt.load(nd, j + G_::NPW, jb, lane);  // prefetch the next group
        const int mine = j + half;
        const bool act = (G_::NPW == 1) || mine < jb;
        const T Wj = (act && apply_W) ? reinterpret_cast<const T *>(nd.W)[mine] : T(1);
        warp_kernel_values<T, D, W>(cur, kslot, ker);
        __syncwarp();
        T accr = T(0), acci = T(0);
        if (act) {
            T k0[L];
#pragma unroll
            for (int q = 0; q < L; q++) k0[q] = (D == 3) ? kh[q] : T(1);
            const int obase = origin_index<G_, D>(cur.r0, cur.r1, cur.r2);
#pragma unroll
            for (int ps = 0; ps < PASSES; ps++) {
                if (coff[ps] >= 0) {
                    const T kab = kh[kab_off[ps] & 0xffff] * kh[kab_off[ps] >> 16];
                    const int idx = obase + coff[ps];
                    const T *pr = tr + idx, *pi = ti + idx;  // the column's run: constant offsets
                    T sr = T(0), si = T(0);
#pragma unroll
                    for (int q0 = 0; q0 < L; q0++) {
                        sr += k0[q0] * pr[q0 * PLANE];
                        si += k0[q0] * pi[q0 * PLANE];
                    }
                    accr += kab * sr;
                    acci += kab * si;
                }
            }
        }
#pragma unroll
        for (int off = G_::LPN / 2; off > 0; off >>= 1) {  // within each node's lanes
            accr += __shfl_xor_sync(0xffffffffu, accr, off);
            acci += __shfl_xor_sync(0xffffffffu, acci, off);
        }
        if (hl == 0 && act) {
            if constexpr (EN) eacc.add(Wj * (accr * accr + acci * acci), T(1));  // W_j |rho_hat_j|^2
            else c_out[mine] = cmake<T2>(accr * Wj, acci * Wj);
        }
        __syncwarp();
        cur = nxt;
    }
    if constexpr (EN) {  // energy-only mode: one compensated partial per CTA
        __syncthreads();
        const double2 tot = energy_block_sum(eacc, reinterpret_cast<double *>(smem_raw));
        if (threadIdx.x == 0) epart[blockIdx.x] = tot;
    }
}

__device__ __forceinline__ void atomic_add_cx(float2 *p, float re, float im) {
    atomicAdd(p, make_float2(re, im));
}
__device__ __forceinline__ void atomic_add_cx(double2 *p, double re, double im) {
    atomicAdd(&p->x, re);
    atomicAdd(&p->y, im);
}

template <typename T, int D, int W>
__global__ void __launch_bounds__(SUB_THREADS) spread_sub_kernel(NodeDesc nd,
                                                                const cx_t<T> *__restrict__ c_in,
                                                                cx_t<T> *__restrict__ H) {
    using T2 = cx_t<T>;
    using G_ = Geo<T, D, W>;
    using F = FixAcc<T>;
    using A = typename F::A;
    constexpr int PASSES = G_::PASSES, L = (D == 3) ? W : 1, PLANE = G_::T1 * G_::T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A *tr = reinterpret_cast<A *>(smem_raw);
    A *ti = tr + G_::NCELL;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int nw = SUB_THREADS / 32;  // the kernels are launched with SUB_THREADS threads
    T *ker = reinterpret_cast<T *>(ti + G_::NCELL) + wid * 6 * MAXW;
    const int4 sb = nd.subs[blockIdx.x];
    const int4 bo = nd.bins[sb.z];
    const int n = nd.n, pad = nd.pad;
    // per-lane constants (see the interpolation kernel)
    int coff[PASSES], kab_off[PASSES], kslot[NodeGroup<T, D, W>::KV];
#pragma unroll
    for (int ps = 0; ps < PASSES; ps++) {
        const int pq = nd.pair_order[ps * G_::LPN + lane % G_::LPN];
        const int qa = pq >> 8, qb = pq & 255;
        coff[ps] = pq >= 0 ? column_offset<G_, D>(qa, qb) : -1;
        kab_off[ps] = (D == 3) ? (MAXW + qa) | ((2 * MAXW + qb) << 16) : qa | ((MAXW + qb) << 16);
    }
#pragma unroll
    for (int v = 0; v < NodeGroup<T, D, W>::KV; v++) kslot[v] = kernel_slot<T, D, W>(lane, v);

    // bound B = max(sum |Re c_j|, sum |Im c_j|) over the subproblem, while the tile is cleared
    T bre = T(0), bim = T(0);
    for (int i = threadIdx.x; i < sb.y; i += blockDim.x) {
        const T2 v = c_in[sb.x + i];
        bre += fabs(v.x);
        bim += fabs(v.y);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        bre += __shfl_xor_sync(0xffffffffu, bre, off);
        bim += __shfl_xor_sync(0xffffffffu, bim, off);
    }
    for (int cell = threadIdx.x; cell < G_::NCELL; cell += blockDim.x) {
        tr[cell] = 0;
        ti[cell] = 0;
    }
    if (lane == 0) {
        ker[0] = bre;  // the warp's kernel table is free until the node loop
        ker[1] = bim;
    }
    __syncthreads();
    T sre = T(0), sim = T(0);
    for (int q = 0; q < nw; q++) {
        const T *kq = reinterpret_cast<T *>(ti + G_::NCELL) + q * 6 * MAXW;
        sre += kq[0];
        sim += kq[1];
    }
    // B to within rounding (<= 1024 terms: a relative 1e-4 in FP32, 1e-13 in FP64); the room
    // above 2^E absorbs it (FP32: int32 cells, 4x; FP64: contributions below 2^51 for the
    // rounding by fused multiply-add, 2x)
    // (fmax drops a NaN operand: a non-finite sum makes the bound NaN explicitly)
    const T bound = (isfinite(sre) && isfinite(sim)) ? fmax(sre, sim) : T(NAN);
    if (!(bound > T(0))) {
        // zero: every c_j of the subproblem is zero, nothing to add.  Non-finite: a c_j has no
        // fixed-point image; a NaN in the grid's first cell (the plane below the stored half,
        // folded into the half by the first inverse pass) reaches every u as it would without
        // the fixed-point accumulation (NaN absorbs any concurrent addition to the cell)
        if (bound != T(0) && threadIdx.x == 0) H[0] = cmake<T2>(T(NAN), T(NAN));
        return;
    }
    int ex = F::E - ilogb(bound) - 1;  // S = 2^ex, S * bound <= 2^E
    if (ex > F::MAXEXP) ex = F::MAXEXP;   // tiny bounds: keep S finite (cells stay < 2^E)
    const T S = (T)ldexp(1.0, ex), inv_s = (T)ldexp(1.0, -ex);
    __syncthreads();  // every warp has read the bound before the tables are overwritten

    int ja, jb;
    warp_chunk(sb, wid, ja, jb);
    const int half = lane / G_::LPN;
    const T *kh = ker + half * 3 * MAXW;
    NodeGroup<T, D, W> cur, nxt;
    T2 c = czero<T2>(), cn = czero<T2>();
    if (ja < jb) {
        cur.load(nd, ja, jb, lane);
        if (ja + half < jb) c = c_in[ja + half];
    }
    for (int j = ja; j < jb; j += G_::NPW) {
        if (j + G_::NPW < jb) {  // prefetch the next group
            nxt.load(nd, j + G_::NPW, jb, lane);
            cn = (j + G_::NPW + half < jb) ? c_in[j + G_::NPW + half] : czero<T2>();
        }
        const bool act = (G_::NPW == 1) || j + half < jb;
        warp_kernel_values<T, D, W>(cur, kslot, ker);
        __syncwarp();
        if (act) {
            T k0[L];
#pragma unroll
            for (int q = 0; q < L; q++) k0[q] = (D == 3) ? kh[q] : T(1);
            const T csr = c.x * S, csi = c.y * S;
            const int obase = origin_index<G_, D>(cur.r0, cur.r1, cur.r2);
#pragma unroll
            for (int ps = 0; ps < PASSES; ps++) {
                if (coff[ps] >= 0) {
                    const T kab = kh[kab_off[ps] & 0xffff] * kh[kab_off[ps] >> 16];
                    const T cr = csr * kab, ci = csi * kab;
                    const int idx = obase + coff[ps];
                    A *pr = tr + idx, *pi = ti + idx;  // the column's run: constant offsets
#pragma unroll
                    for (int q0 = 0; q0 < L; q0++) {
                        F::add(pr + q0 * PLANE, F::mulq(cr, k0[q0]));
                        F::add(pi + q0 * PLANE, F::mulq(ci, k0[q0]));
                    }
                }
            }
        }
        __syncwarp();
        cur = nxt;
        c = cn;
    }
    __syncthreads();

    const int slot = bo.w;
    const int nplanes = n / 2 + 1 + 2 * pad;
    if (D == 3 && slot < 0) {
        // by (axis-1, axis-2) column, as the interpolation's tile load: wrapped offsets once,
        // then the planes of the extended grid at a constant stride
        const int64_t nn = (int64_t)n * n;
        for (int col = threadIdx.x; col < PLANE; col += blockDim.x) {
            const int a1 = col / G_::T2, a2 = col - a1 * G_::T2;
            const int64_t gb = (int64_t)wrap1(bo.y + a1, n) * n + wrap1(bo.z + a2, n);
#pragma unroll
            for (int a0 = 0; a0 < G_::T0; a0++) {
                const A qr = tr[a0 * PLANE + col], qi = ti[a0 * PLANE + col];
                const int pl = bo.x + a0 + pad;
                if ((qr == 0 && qi == 0) || pl < 0 || pl >= nplanes) continue;
                atomic_add_cx(H + pl * nn + gb, (T)qr * inv_s, (T)qi * inv_s);
            }
        }
        return;
    }
    for (int cell = threadIdx.x; cell < G_::NCELL; cell += blockDim.x) {
        const A qr = tr[cell], qi = ti[cell];
        if (qr == 0 && qi == 0) continue;
        if (slot >= 0) {  // crowded bin: FP64 sum across its subproblems (exact: q / 2^ex)
            const double is = ldexp(1.0, -ex);
            atomic_add_cx(nd.crowd + (int64_t)slot * G_::NCELL + cell, (double)qr * is, (double)qi * is);
            continue;
        }
        int a0, a1, a2;
        cell_coords<G_>(cell, a0, a1, a2);
        const int pl = bo.x + a0 + pad;
        if (pl < 0 || pl >= nplanes) continue;  // outside every stencil: the cell is zero
        const int64_t g = (D == 3)
            ? ((int64_t)pl * n + wrap1(bo.y + a1, n)) * n + wrap1(bo.z + a2, n)
            : (int64_t)pl * n + wrap1(bo.y + a1, n);
        atomic_add_cx(H + g, (T)qr * inv_s, (T)qi * inv_s);
    }
}

template <typename T, int D, int W>
static cudaError_t launch_interp_w(const NodeDesc &nd, const void *G, void *c_out, int apply_W,
                                   double2 *epart, size_t smem, cudaStream_t s) {
    if (epart) {
        cudaError_t e = cudaFuncSetAttribute(interp_sub_kernel<T, D, W, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        interp_sub_kernel<T, D, W, true><<<(unsigned)nd.nsub, SUB_THREADS, smem, s>>>(
            nd, (const cx_t<T> *)G, (cx_t<T> *)c_out, apply_W, epart);
    } else {
        cudaError_t e = cudaFuncSetAttribute(interp_sub_kernel<T, D, W, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        interp_sub_kernel<T, D, W, false><<<(unsigned)nd.nsub, SUB_THREADS, smem, s>>>(
            nd, (const cx_t<T> *)G, (cx_t<T> *)c_out, apply_W, nullptr);
    }
    return cudaGetLastError();
}

template <typename T, int D, int W>
static cudaError_t launch_spread_w(const NodeDesc &nd, const void *c_in, void *H, size_t smem,
                                   cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(spread_sub_kernel<T, D, W>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    spread_sub_kernel<T, D, W><<<(unsigned)nd.nsub, SUB_THREADS, smem, s>>>(
        nd, (const cx_t<T> *)c_in, (cx_t<T> *)H);
    return cudaGetLastError();
}

// Adds the FP64 tiles of the crowded bins into the extended spread grid (one CTA per tile).
template <typename T, int D>
__global__ void __launch_bounds__(SUB_THREADS) crowd_merge_kernel(NodeDesc nd, cx_t<T> *__restrict__ H) {
    const int T1 = nd.T[1], T2n = (D == 3) ? nd.T[2] : 1;
    const int ncell = nd.T[0] * T1 * T2n;
    const int slot = blockIdx.x;
    const int4 bo = nd.bins[nd.crowd_bin[slot]];
    const int n = nd.n, pad = nd.pad;
    const int nplanes = n / 2 + 1 + 2 * pad;
    const double2 *src = nd.crowd + (int64_t)slot * ncell;
    for (int cell = threadIdx.x; cell < ncell; cell += blockDim.x) {
        const double2 v = src[cell];
        if (v.x == 0.0 && v.y == 0.0) continue;
        const int a0 = cell / (T1 * T2n), rem = cell - a0 * T1 * T2n;
        const int a1 = rem / T2n, a2 = rem - a1 * T2n;
        const int pl = bo.x + a0 + pad;
        if (pl < 0 || pl >= nplanes) continue;
        const int64_t g = (D == 3)
            ? ((int64_t)pl * n + wrap1(bo.y + a1, n)) * n + wrap1(bo.z + a2, n)
            : (int64_t)pl * n + wrap1(bo.y + a1, n);
        atomic_add_cx(H + g, (T)v.x, (T)v.y);
    }
}

template <typename T, int D>
cudaError_t launch_crowd_merge_d(const NodeDesc &nd, void *H, cudaStream_t s) {
    if (nd.ncrowd == 0) return cudaSuccess;
    crowd_merge_kernel<T, D><<<(unsigned)nd.ncrowd, SUB_THREADS, 0, s>>>(nd, (cx_t<T> *)H);
    return cudaGetLastError();
}

#define NLINT_W_SWITCH(CALL)                                                   \
    switch (nd.w) {                                                            \
        case 2: return CALL(2);   case 3: return CALL(3);                      \
        case 4: return CALL(4);   case 5: return CALL(5);                      \
        case 6: return CALL(6);   case 7: return CALL(7);                      \
        case 8: return CALL(8);   case 9: return CALL(9);                      \
        case 10: return CALL(10); case 11: return CALL(11);                    \
        case 12: return CALL(12); case 13: return CALL(13);                    \
        case 14: return CALL(14); case 15: return CALL(15);                    \
        case 16: return CALL(16);                                              \
        default: return cudaErrorInvalidValue;                                 \
    }

template <typename T, int D>
cudaError_t launch_interp_d(const NodeDesc &nd, const void *G, void *c_out, int apply_W,
                            double2 *epart, cudaStream_t s) {
    if (nd.nsub == 0) return cudaSuccess;
    const size_t sm = node_smem(nd, sizeof(T) == 4 ? NLINT_FP32 : NLINT_FP64);
#define NLINT_CALL_I(WW) launch_interp_w<T, D, WW>(nd, G, c_out, apply_W, epart, sm, s)
    NLINT_W_SWITCH(NLINT_CALL_I)
#undef NLINT_CALL_I
}

template <typename T, int D>
cudaError_t launch_spread_d(const NodeDesc &nd, const void *c_in, void *H, cudaStream_t s) {
    if (nd.nsub == 0) return cudaSuccess;
    const size_t sm = node_smem(nd, sizeof(T) == 4 ? NLINT_FP32 : NLINT_FP64);
#define NLINT_CALL_S(WW) launch_spread_w<T, D, WW>(nd, c_in, H, sm, s)
    NLINT_W_SWITCH(NLINT_CALL_S)
#undef NLINT_CALL_S
}

#define NLINT_NODE_KERNELS_INSTANTIATE(T, D)                                                    \
    template cudaError_t launch_interp_d<T, D>(const NodeDesc &, const void *, void *, int,      \
                                               double2 *, cudaStream_t);                       \
    template cudaError_t launch_spread_d<T, D>(const NodeDesc &, const void *, void *,           \
                                               cudaStream_t);                                  \
    template cudaError_t launch_crowd_merge_d<T, D>(const NodeDesc &, void *, cudaStream_t);

}  // namespace nlint
