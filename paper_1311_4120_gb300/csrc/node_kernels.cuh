// Type-2 interpolation with the multiply by W_j, and type-1 spreading (steps a3, a4 and a5 of
// the path; Algorithm 1, eq. 3.2 and eq. 3.7), templated on the stencil width and the bin
// shape so that every loop over the stencil is unrolled and every tile index is a
// compile-time product.
//
// Spreading function: the "exponential of semicircle" of Barnett, Magland and af Klinteberg
// (SIAM J. Sci. Comput. 2019), phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1, with
// z = (l - g) / (w/2) for fine cell l and node position g in fine-cell units.  FP64 plans
// evaluate phi for every node and axis once on the host, in FP64, and the kernels read those
// values; FP32 kernels evaluate phi from each node's fractional offsets in registers (a
// 16-byte record per node instead of d w stored values) and hand the values to the lanes
// that need them by warp shuffles.
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
#include <cstring>

namespace nlint {

static constexpr int MAXW = NODE_MAXW;
static constexpr int SUB_THREADS = NODE_THREADS;

template <typename T, int D, int W, int BS>
struct Geo {
    static constexpr bool F64 = sizeof(T) == 8;
    static constexpr int B0 = bin_dim(D, BS, 0), B1 = bin_dim(D, BS, 1);
    static constexpr int B2 = (D == 3) ? bin_dim(D, BS, 2) : 1;
    static constexpr int T0 = B0 + W - 1, T1 = B1 + W - 1, T2 = (D == 3) ? B2 + W - 1 : 1;
    // shared layout: axis-2 rows of P2 >= T2 cells (padded against bank conflicts), planes of
    // T1 rows; cells with axis-2 offset >= T2 are padding that no stencil touches
    static constexpr int P2 = (D == 3) ? tile_pitch(F64, D, W, BS) : 1;
    static constexpr int PLANE = (D == 3) ? T1 * P2 : T1;
    static constexpr int NCELL = T0 * PLANE;
    static constexpr int PAIRS = W * W;  // stencil columns per node
    // lanes per node: 16 (two nodes per warp) when that wastes fewer lane slots, else 32
    static constexpr int LPN = node_lanes(W);
    static constexpr int NPW = 32 / LPN;                 // nodes per warp iteration
    static constexpr int PASSES = (PAIRS + LPN - 1) / LPN;
    // resident CTAs of the FP32 spreading that the shared memory allows (its two int32 planes
    // and the per-CTA reserve of the 228 KB per SM), at most 4 (w <= 8) or 2 (wider stencils,
    // whose per-lane state needs more than 64 registers): its register budget follows
    static constexpr int SPREAD_MINB_RAW = (228 * 1024) / (NCELL * 8 + 1024 + 256);
    static constexpr int SPREAD_MINB_CAP = W <= 8 ? 4 : 2;
    static constexpr int SPREAD_MINB = SPREAD_MINB_RAW < 1 ? 1
                                     : (SPREAD_MINB_RAW > SPREAD_MINB_CAP ? SPREAD_MINB_CAP : SPREAD_MINB_RAW);
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

// ---------------------------------------------------------------- shared by both precisions

// Decompose a tile cell into its per-axis offsets.
template <typename G_>
__device__ __forceinline__ void cell_coords(int cell, int &a0, int &a1, int &a2) {
    a0 = cell / G_::PLANE;
    const int rem = cell - a0 * G_::PLANE;
    a1 = rem / G_::P2;
    a2 = rem - a1 * G_::P2;
}

// Tile offset of stencil column (qa, qb) for the origin (r0, r1, r2), axis-0 run start:
// origin_index(r0, r1, r2) + column_offset(qa, qb).
template <typename G_, int D>
__device__ __forceinline__ int origin_index(int r0, int r1, int r2) {
    return (D == 3) ? (r0 * G_::T1 + r1) * G_::P2 + r2 : r0 * G_::T1 + r1;
}
template <typename G_, int D>
__device__ __forceinline__ int column_offset(int qa, int qb) {
    return (D == 3) ? qa * G_::P2 + qb : qa * G_::T1 + qb;
}

// Each warp owns a contiguous run of its subproblem's nodes.
// (32-bit: a subproblem holds at most 2^20 nodes; the warp count is the compile-time
// SUB_THREADS / 32, so the division is a shift.)
__device__ __forceinline__ void warp_chunk(int4 sb, int wid, int &ja, int &jb) {
    constexpr int NW = SUB_THREADS / 32;
    ja = sb.x + (sb.y * wid) / NW;
    jb = sb.x + (sb.y * (wid + 1)) / NW;
}


// Stages the bin's tile of G (T0 x T1 (x T2) cells from the bin origin) in shared memory as
// real and imaginary planes.  The common case (axis-0 planes inside the stored half) goes by
// (axis-1, axis-2) column: its wrapped offsets and base index once, then the T0 planes at a
// constant stride; tiles that reach outside the stored half read the mirror by conjugation.
template <typename T, typename G_, int D>
__device__ __forceinline__ void stage_tile(const cx_t<T> *__restrict__ G, int4 bo, int n, T *tr, T *ti) {
    using T2 = cx_t<T>;
    constexpr int PLANE = G_::PLANE;
    const bool inside = bo.x >= 0 && bo.x + G_::T0 - 1 <= n / 2;
    if (D == 3 && inside) {
        const int64_t nn = (int64_t)n * n;
        for (int col = threadIdx.x; col < PLANE; col += blockDim.x) {
            const int a1 = col / G_::P2, a2 = col - a1 * G_::P2;
            if (a2 >= G_::T2) continue;  // row padding
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
            if (D == 3 && a2 >= G_::T2) continue;  // row padding
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
}

__device__ __forceinline__ void atomic_add_cx(float2 *p, float re, float im) {
    atomicAdd(p, make_float2(re, im));
}
__device__ __forceinline__ void atomic_add_cx(double2 *p, double re, double im) {
    atomicAdd(&p->x, re);
    atomicAdd(&p->y, im);
}

// Adds a spreading tile of fixed-point sums (multiples of 2^-ex) into the extended spread grid
// H+ (planes -pad .. n/2 + pad of axis 0) with global atomics, or, for a crowded bin (bo.w is
// its crowd slot), exactly into its FP64 tile.  Zero cells are skipped.
template <typename T, typename G_, int D, typename A>
__device__ __forceinline__ void flush_tile(const A *tr, const A *ti, int4 bo, const NodeDesc &nd, int ex,
                                           cx_t<T> *__restrict__ H) {
    constexpr int PLANE = G_::PLANE;
    const int n = nd.n, pad = nd.pad, slot = bo.w;
    const int nplanes = n / 2 + 1 + 2 * pad;
    const T inv_s = (T)ldexp(1.0, -ex);
    if constexpr (D == 3 && sizeof(T) == 4) {
        if (slot < 0 && (bo.z & 1) == 0) {
            // FP32: two adjacent axis-2 cells per 16-byte vector atomic.  The bin origin along
            // axis 2 is even (the plan aligns its bins), n is even, so a pair starts at an even
            // grid index: 16-byte aligned and never split by the periodic wrap
            const int64_t nn = (int64_t)n * n;
            constexpr int PPR = (G_::T2 + 1) / 2;  // cell pairs per row
            for (int cp = threadIdx.x; cp < G_::T1 * PPR; cp += blockDim.x) {
                const int a1 = cp / PPR, a2 = 2 * (cp - a1 * PPR);
                const bool two = a2 + 1 < G_::T2;
                const int64_t gb = (int64_t)wrap1(bo.y + a1, n) * n + wrap1(bo.z + a2, n);
#pragma unroll 4
                for (int a0 = 0; a0 < G_::T0; a0++) {
                    const int c0 = a0 * PLANE + a1 * G_::P2 + a2;
                    const A qr0 = tr[c0], qi0 = ti[c0];
                    const A qr1 = two ? tr[c0 + 1] : 0, qi1 = two ? ti[c0 + 1] : 0;
                    const int pl = bo.x + a0 + pad;
                    if ((qr0 == 0 && qi0 == 0 && qr1 == 0 && qi1 == 0) || pl < 0 || pl >= nplanes) continue;
                    atomicAdd(reinterpret_cast<float4 *>(H + pl * nn + gb),
                              make_float4((T)qr0 * inv_s, (T)qi0 * inv_s, (T)qr1 * inv_s, (T)qi1 * inv_s));
                }
            }
            return;
        }
    }
    if (D == 3 && slot < 0) {
        // by (axis-1, axis-2) column, as the tile load: wrapped offsets once, then the planes of
        // the extended grid at a constant stride
        const int64_t nn = (int64_t)n * n;
        for (int col = threadIdx.x; col < PLANE; col += blockDim.x) {
            const int a1 = col / G_::P2, a2 = col - a1 * G_::P2;
            if (a2 >= G_::T2) continue;  // row padding (never added to)
            const int64_t gb = (int64_t)wrap1(bo.y + a1, n) * n + wrap1(bo.z + a2, n);
#pragma unroll 4
            for (int a0 = 0; a0 < G_::T0; a0++) {
                const A qr = tr[a0 * PLANE + col], qi = ti[a0 * PLANE + col];
                const int pl = bo.x + a0 + pad;
                if ((qr == 0 && qi == 0) || pl < 0 || pl >= nplanes) continue;
                atomic_add_cx(H + pl * nn + gb, (T)qr * inv_s, (T)qi * inv_s);
            }
        }
        return;
    }
    constexpr int TCELL = G_::T0 * G_::T1 * G_::T2;  // unpadded cells: the crowd tile's layout
    for (int cell = threadIdx.x; cell < G_::NCELL; cell += blockDim.x) {
        const A qr = tr[cell], qi = ti[cell];
        if (qr == 0 && qi == 0) continue;  // (row padding is never added to: always zero)
        int a0, a1, a2;
        cell_coords<G_>(cell, a0, a1, a2);
        if (slot >= 0) {  // crowded bin: FP64 sum across its subproblems (exact: q / 2^ex)
            const double is = ldexp(1.0, -ex);
            const int tc = (a0 * G_::T1 + a1) * G_::T2 + a2;
            atomic_add_cx(nd.crowd + (int64_t)slot * TCELL + tc, (double)qr * is, (double)qi * is);
            continue;
        }
        const int pl = bo.x + a0 + pad;
        if (pl < 0 || pl >= nplanes) continue;  // outside every stencil: the cell is zero
        const int64_t g = (D == 3)
            ? ((int64_t)pl * n + wrap1(bo.y + a1, n)) * n + wrap1(bo.z + a2, n)
            : (int64_t)pl * n + wrap1(bo.y + a1, n);
        atomic_add_cx(H + g, (T)qr * inv_s, (T)qi * inv_s);
    }
}

// Fixed-point accumulation of the spreading tile.  Shared-memory floating-point atomics are
// several times slower than integer ones on this GPU, so each CTA adds integer multiples of
// 1/S: S = 2^(E - ceil(log2 B)) with B >= max(sum_j |Re c_j|, sum_j |Im c_j|) over the
// subproblem (every cell sum and every contribution is at most B, since phi <= 1), E = 29 for
// FP32 (int32 cells) and 50 for FP64 (int64 cells), so no cell can overflow.  Each
// contribution is rounded to 1/S <= 2^-E B (FP32: 2^-29 B, finer than FP32 rounding of the
// largest cells; FP64: 2^-50 B); the integer sums are exact, so a tile does not depend on the
// order of its additions.  FP64 rounds with one fused multiply-add: a * b + 1.5 * 2^52 lies in
// [2^52, 2^53) for |a * b| < 2^51, where the spacing of doubles is 1, so its low mantissa bits
// are a * b rounded to the nearest integer (the classic magic-number conversion) -- one
// operation on the FP64 units, which bound the FP64 path, instead of a multiply and a convert.
// FP32 3D uses the same conversion in single precision where a contribution is within its
// range (see fmaq and spread_f32_kernel).
template <typename T> struct FixAcc;
template <> struct FixAcc<float> {
    using A = int;
    static constexpr int E = 29, MAXEXP = 126;
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

// Scale exponent of a spreading CTA: reads the subproblem's c values, sums |Re| and |Im| over
// the CTA (the bound B above), clears the tile and returns ex with S = 2^ex (S B <= 2^E), or
// INT_MIN when the subproblem adds nothing (all c zero) or a c is not finite (then the first
// cell of H+ is set to NaN, which the first inverse pass folds into every output, as a
// floating-point accumulation would).  `red` is 2 * (SUB_THREADS / 32) entries of shared
// scratch.
template <typename T, typename A, int NCELL, int E, int MAXEXP>
__device__ __forceinline__ int spread_scale(const cx_t<T> *__restrict__ c_in, int4 sb, A *tr, A *ti,
                                            T *red, cx_t<T> *__restrict__ H) {
    using T2 = cx_t<T>;
    constexpr int nw = SUB_THREADS / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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
    for (int cell = threadIdx.x; cell < NCELL; cell += blockDim.x) {
        tr[cell] = 0;
        ti[cell] = 0;
    }
    if (lane == 0) {
        red[2 * wid] = bre;
        red[2 * wid + 1] = bim;
    }
    __syncthreads();
    T sre = T(0), sim = T(0);
    for (int q = 0; q < nw; q++) {
        sre += red[2 * q];
        sim += red[2 * q + 1];
    }
    // B to within rounding (<= 1024 terms: a relative 1e-4 in FP32, 1e-13 in FP64); the room
    // above 2^E absorbs it (FP32: int32 cells, 4x; FP64: contributions below 2^51 for the
    // rounding by fused multiply-add, 2x)
    // (fmax drops a NaN operand: a non-finite sum makes the bound NaN explicitly)
    const T bound = (isfinite(sre) && isfinite(sim)) ? fmax(sre, sim) : T(NAN);
    if (!(bound > T(0))) {
        if (bound != T(0) && threadIdx.x == 0) H[0] = cmake<T2>(T(NAN), T(NAN));
        return INT_MIN;
    }
    int ex = E - ilogb(bound) - 1;  // S = 2^ex, S * bound <= 2^E
    if (ex > MAXEXP) ex = MAXEXP;    // tiny bounds: keep S finite (cells stay < 2^E)
    return ex;
}

// ------------------------------------------------- FP64: stencil values precomputed per node

// A warp works on NPW = 32 / LPN nodes at a time (one per LPN-lane group): per node its lanes
// share the w*w stencil columns, and the nodes share the warp's per-node work (loads, shuffle
// reductions).  NodeGroup holds this lane's view: the stencil origin of its group's node
// (relative to the bin) and its share of the group's NPW*D*w kernel values, which the plan
// computed once (the nodes are fixed).
template <typename T, int D, int W>
struct NodeGroup {
    static constexpr int LPN = Geo<T, D, W, 1>::LPN, NPW = Geo<T, D, W, 1>::NPW;
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

template <typename T, int D, int W, int BS, bool EN>
__global__ void __launch_bounds__(SUB_THREADS) interp_sub_kernel(NodeDesc nd,
                                                                const cx_t<T> *__restrict__ G,
                                                                cx_t<T> *__restrict__ c_out,
                                                                int apply_W,
                                                                double2 *__restrict__ epart) {
    pdl_wait();  // (launched by launch_pdl)
    pdl_trigger();
    using T2 = cx_t<T>;
    using G_ = Geo<T, D, W, BS>;
    constexpr int PASSES = G_::PASSES, L = (D == 3) ? W : 1, PLANE = G_::PLANE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the tile as real and imaginary planes (measured faster than interleaved complex, whose
    // one 8-byte load per stencil cell cost registers and resident CTAs)
    T *tr = reinterpret_cast<T *>(smem_raw);
    T *ti = tr + G_::NCELL;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T *ker = ti + G_::NCELL + wid * 6 * MAXW;
    const int4 sb = nd.subs[blockIdx.x];
    const int4 bo = nd.bins[sb.z];
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

    stage_tile<T, G_, D>(G, bo, nd.n, tr, ti);
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

template <typename T, int D, int W, int BS>
__global__ void __launch_bounds__(SUB_THREADS) spread_sub_kernel(NodeDesc nd,
                                                                const cx_t<T> *__restrict__ c_in,
                                                                cx_t<T> *__restrict__ H) {
    pdl_wait();  // (launched by launch_pdl)
    pdl_trigger();
    using T2 = cx_t<T>;
    using G_ = Geo<T, D, W, BS>;
    using F = FixAcc<T>;
    using A = typename F::A;
    constexpr int PASSES = G_::PASSES, L = (D == 3) ? W : 1, PLANE = G_::PLANE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A *tr = reinterpret_cast<A *>(smem_raw);
    A *ti = tr + G_::NCELL;
    __shared__ T red[2 * (SUB_THREADS / 32)];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T *ker = reinterpret_cast<T *>(ti + G_::NCELL) + wid * 6 * MAXW;
    const int4 sb = nd.subs[blockIdx.x];
    const int4 bo = nd.bins[sb.z];
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

    const int ex = spread_scale<T, A, G_::NCELL, F::E, F::MAXEXP>(c_in, sb, tr, ti, red, H);
    if (ex == INT_MIN) return;
    const T S = (T)ldexp(1.0, ex);

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
    flush_tile<T, G_, D, A>(tr, ti, bo, nd, ex, H);
}

// ------------------------------------------ FP32: stencil values evaluated from the offsets

// phi(z) = exp(beta (sqrt(1 - z^2) - 1)) for |z| <= 1, written as exp(-beta z^2 / (1 +
// sqrt(1 - z^2))): the second form has no cancellation next to z = 0, where phi is largest, so
// its FP32 rounding stays a few ulps relative for the values that matter.  1 - z^2 is clamped
// at 0, so a z that rounds onto +-1 gives exp(-beta), the limit from inside.  The truncated
// function jumps from exp(-beta) to 0 at |z| = 1 (1e-4 at w = 4, 1e-7 at w = 7): which cells
// take the jump is decided exactly, from the offsets (see F32Lane::values), never by rounding.
__device__ __forceinline__ float es_phi_f32(float z, float beta) {
    const float z2 = z * z;
    const float t = fmaxf(1.0f - z2, 0.0f);
    const float s = t * rsqrtf(fmaxf(t, 1e-30f));
    return __expf(__fdividef(-beta * z2, 1.0f + s));
}

// Value slot t of the warp's group (slot t lives in register t / 32 of lane t % 32).
template <int KV, typename V>
__device__ __forceinline__ V shfl_slot(const V (&v)[KV], int t) {
    V r = __shfl_sync(0xffffffffu, v[0], t & 31);
#pragma unroll
    for (int k = 1; k < KV; k++) {
        const V x = __shfl_sync(0xffffffffu, v[k], t & 31);
        if ((t >> 5) == k) r = x;
    }
    return r;
}

// round(a b) for |a b| <= 2^22, by one fused multiply-add: a b + 1.5 * 2^23 lies in [2^23, 2^24],
// where the spacing of floats is 1, so the sum is rounded once, to the nearest integer, and its
// bit pattern minus that of 1.5 * 2^23 is that integer (the classic magic-number conversion in
// single precision; no float-to-integer conversion instruction per stencil cell)
__device__ __forceinline__ int fmaq(float a, float b) {
    return __float_as_int(fmaf(a, b, 12582912.0f)) - 0x4B400000;
}
static constexpr float FMAQ_MAX = 4194304.0f;  // 2^22

// Adds one stencil column of one node, or of two nodes with the same origin, into the
// fixed-point tile along axis 0 (FAST: every weight within 2^22, contributions by fmaq; else by
// the rounded product and a conversion).
template <bool FAST>
__device__ __forceinline__ int fix_contrib(float w, float k) {
    if constexpr (FAST) return fmaq(w, k);
    else return __float2int_rn(w * k);
}
template <bool FAST, int L, int PLANE>
__device__ __forceinline__ void add_column(int *pr, int *pi, float wr, float wi, const float (&k)[L]) {
#pragma unroll
    for (int q0 = 0; q0 < L; q0++) {
        atomicAdd(pr + q0 * PLANE, fix_contrib<FAST>(wr, k[q0]));
        atomicAdd(pi + q0 * PLANE, fix_contrib<FAST>(wi, k[q0]));
    }
}
template <bool FAST, int L, int PLANE>
__device__ __forceinline__ void add_column2(int *pr, int *pi, float wr, float wi, const float (&k)[L],
                                            float wr2, float wi2, const float (&k2)[L]) {
#pragma unroll
    for (int q0 = 0; q0 < L; q0++) {
        atomicAdd(pr + q0 * PLANE, fix_contrib<FAST>(wr, k[q0]) + fix_contrib<FAST>(wr2, k2[q0]));
        atomicAdd(pi + q0 * PLANE, fix_contrib<FAST>(wi, k[q0]) + fix_contrib<FAST>(wi2, k2[q0]));
    }
}

// Sums four per-lane values over the warp with five shuffles (a transposed butterfly: the
// first two steps exchange halves of the value set, the last three sum one value): afterwards
// lanes 0-7 hold the total of v0, 8-15 of v1, 16-23 of v2, 24-31 of v3.
__device__ __forceinline__ float warp_sum4(float v0, float v1, float v2, float v3, int lane) {
    const bool h16 = lane & 16, h8 = lane & 8;
    float k0 = h16 ? v2 : v0, k1 = h16 ? v3 : v1;
    k0 += __shfl_xor_sync(0xffffffffu, h16 ? v0 : v2, 16);
    k1 += __shfl_xor_sync(0xffffffffu, h16 ? v1 : v3, 16);
    float k = h8 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    return k;
}

// FP32 per-lane constants: this lane's value slots (node of the group, axis, and the cell's
// part of z), and its columns' tile offsets and value slots.
template <int D, int W, int BS>
struct F32Lane {
    using G_ = Geo<float, D, W, BS>;
    static constexpr int LPN = G_::LPN, NPW = G_::NPW, DW = D * W, PASSES = G_::PASSES;
    static constexpr int NKV = NPW * DW, KV = (NKV + 31) / 32;
    int vnode[KV], vax[KV];
    float vc[KV];                // (q + 1 - w/2) (2 / w) of the slot's cell q
    bool vfirst[KV];             // the slot's cell is the first of its axis (q = 0)
    int coff[PASSES], sa[PASSES], sb[PASSES];
    __device__ __forceinline__ void init(const int16_t *__restrict__ pair_order, int lane) {
        const int half = lane / LPN, hl = lane % LPN;
#pragma unroll
        for (int v = 0; v < KV; v++) {
            const int t = lane + 32 * v;
            if (t < NKV) {
                const int h = t / DW, rem = t - h * DW, a = rem / W, q = rem - a * W;
                vnode[v] = h;
                vax[v] = a;
                vc[v] = ((float)q + 1.0f - 0.5f * (float)W) * (2.0f / (float)W);
                vfirst[v] = q == 0;
            } else {
                vnode[v] = -1;
                vax[v] = 0;
                vc[v] = 0.0f;
                vfirst[v] = false;
            }
        }
#pragma unroll
        for (int ps = 0; ps < PASSES; ps++) {
            const int pq = pair_order[ps * LPN + hl];
            const int qa = pq >= 0 ? (pq >> 8) : 0, qb = pq >= 0 ? (pq & 255) : 0;
            coff[ps] = pq >= 0 ? column_offset<G_, D>(qa, qb) : -1;
            sa[ps] = half * DW + (D == 3 ? W : 0) + qa;
            sb[ps] = half * DW + (D == 3 ? 2 * W : W) + qb;
        }
    }
    // this lane's stencil values of nodes j .. j + NPW - 1 (those below jb); `me` is the record
    // of node j + lane / LPN, which serves every slot when NPW = 1.  With u in (0, 1], only the
    // first cell can reach |z| = 1, exactly when u = 1; the plan stores u = 1 only for nodes
    // whose FP64 offset is exactly w/2 (the FP64 plans' values are then 0 too) and rounds every
    // other u below 1, so both precisions zero the same cells
    __device__ __forceinline__ void values(const int4 *__restrict__ pos, int j, int jb, int4 me,
                                           float beta, float (&phv)[KV]) const {
#pragma unroll
        for (int v = 0; v < KV; v++) {
            float val = 0.0f;
            const int nn = j + vnode[v];
            if (vnode[v] >= 0 && nn < jb) {
                const int4 r = (NPW == 1) ? me : pos[nn];
                const float u = __int_as_float(vax[v] == 0 ? r.y : (vax[v] == 1 ? r.z : r.w));
                if (!(vfirst[v] && u >= 1.0f)) val = es_phi_f32(fmaf(-u, 2.0f / (float)W, vc[v]), beta);
            }
            phv[v] = val;
        }
    }
};

template <int D, int W, int BS, bool EN>
__global__ void __launch_bounds__(SUB_THREADS) interp_f32_kernel(NodeDesc nd, const float2 *__restrict__ G,
                                                                float2 *__restrict__ c_out, int apply_W,
                                                                double2 *__restrict__ epart) {
    pdl_wait();  // (launched by launch_pdl)
    pdl_trigger();
    using G_ = Geo<float, D, W, BS>;
    using LN = F32Lane<D, W, BS>;
    constexpr int PASSES = G_::PASSES, L = (D == 3) ? W : 1, PLANE = G_::PLANE;
    constexpr int LPN = G_::LPN, NPW = G_::NPW, KV = LN::KV, DW = D * W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tr = reinterpret_cast<float *>(smem_raw);
    float *ti = tr + G_::NCELL;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int4 sb = nd.subs[blockIdx.x];
    const int4 bo = nd.bins[sb.z];
    LN ln;
    ln.init(nd.pair_order_i, lane);
    stage_tile<float, G_, D>(G, bo, nd.n, tr, ti);
    __syncthreads();

    int ja, jb;
    warp_chunk(sb, wid, ja, jb);
    const int half = lane / LPN, hl = lane % LPN;
    const int4 *__restrict__ pos = nd.pos;
    const float *__restrict__ Wv = reinterpret_cast<const float *>(nd.W);
    const float beta = (float)nd.beta;
    EAcc<float> eacc;
    if constexpr (LPN == 32 && D == 3) {
        // Two nodes per iteration (A = j, B = j + 1): both nodes' stencil values come from one
        // evaluation pass over the lanes, their four sums are reduced together (warp_sum4), and
        // when they share a stencil origin (about half of the pairs after the plan's sort by
        // origin) each tile value is loaded once for both.
        int4 rA_n = make_int4(0, 0, 0, 0), rB_n = make_int4(0, 0, 0, 0);
        float WA_n = 1.0f, WB_n = 1.0f;
        if (ja < jb) {
            rA_n = pos[ja];
            if (apply_W) WA_n = Wv[ja];
        }
        if (ja + 1 < jb) {
            rB_n = pos[ja + 1];
            if (apply_W) WB_n = Wv[ja + 1];
        }
        for (int j = ja; j < jb; j += 2) {
            const bool hasB = j + 1 < jb;
            const int4 rA = rA_n, rB = rB_n;
            const float WA = WA_n, WB = WB_n;
            if (j + 2 < jb) {
                rA_n = pos[j + 2];
                if (apply_W) WA_n = Wv[j + 2];
            }
            if (j + 3 < jb) {
                rB_n = pos[j + 3];
                if (apply_W) WB_n = Wv[j + 3];
            }
            float phA[KV], phB[KV];
            ln.values(pos, j, jb, rA, beta, phA);
            ln.values(pos, j + 1, jb, rB, beta, phB);
            float kA[L], kB[L];
#pragma unroll
            for (int q = 0; q < L; q++) {
                kA[q] = shfl_slot<KV>(phA, q);
                kB[q] = shfl_slot<KV>(phB, q);
            }
            const int oA = origin_index<G_, D>(rA.x & 255, (rA.x >> 8) & 255, (rA.x >> 16) & 255);
            const int oB = origin_index<G_, D>(rB.x & 255, (rB.x >> 8) & 255, (rB.x >> 16) & 255);
            const bool same = hasB && rA.x == rB.x;  // the same for every lane
            float aAr = 0.0f, aAi = 0.0f, aBr = 0.0f, aBi = 0.0f;
#pragma unroll
            for (int ps = 0; ps < PASSES; ps++) {
                const float kabA = shfl_slot<KV>(phA, ln.sa[ps]) * shfl_slot<KV>(phA, ln.sb[ps]);
                const float kabB = shfl_slot<KV>(phB, ln.sa[ps]) * shfl_slot<KV>(phB, ln.sb[ps]);
                if (ln.coff[ps] >= 0) {
                    const float *prA = tr + oA + ln.coff[ps], *piA = ti + oA + ln.coff[ps];
                    float sAr = 0.0f, sAi = 0.0f, sBr = 0.0f, sBi = 0.0f;
                    if (same) {
#pragma unroll
                        for (int q0 = 0; q0 < L; q0++) {
                            const float gr = prA[q0 * PLANE], gi = piA[q0 * PLANE];
                            sAr = fmaf(kA[q0], gr, sAr);
                            sAi = fmaf(kA[q0], gi, sAi);
                            sBr = fmaf(kB[q0], gr, sBr);
                            sBi = fmaf(kB[q0], gi, sBi);
                        }
                    } else {
                        const float *prB = tr + oB + ln.coff[ps], *piB = ti + oB + ln.coff[ps];
#pragma unroll
                        for (int q0 = 0; q0 < L; q0++) {
                            sAr = fmaf(kA[q0], prA[q0 * PLANE], sAr);
                            sAi = fmaf(kA[q0], piA[q0 * PLANE], sAi);
                        }
                        if (hasB) {
#pragma unroll
                            for (int q0 = 0; q0 < L; q0++) {
                                sBr = fmaf(kB[q0], prB[q0 * PLANE], sBr);
                                sBi = fmaf(kB[q0], piB[q0 * PLANE], sBi);
                            }
                        }
                    }
                    aAr = fmaf(kabA, sAr, aAr);
                    aAi = fmaf(kabA, sAi, aAi);
                    aBr = fmaf(kabB, sBr, aBr);
                    aBi = fmaf(kabB, sBi, aBi);
                }
            }
            // lane 0: Re A, lane 8: Im A, lane 16: Re B, lane 24: Im B
            const float tot = warp_sum4(aAr, aAi, aBr, aBi, lane);
            const bool isB = lane & 16;
            const int node = j + (isB ? 1 : 0);
            const float Wn = isB ? WB : WA;
            if constexpr (EN) {
                const float im = __shfl_xor_sync(0xffffffffu, tot, 8);
                if ((lane & 15) == 0 && (!isB || hasB)) eacc.add(Wn * (tot * tot + im * im), 1.0f);
            } else {
                if ((lane & 7) == 0 && (!isB || hasB))
                    reinterpret_cast<float *>(c_out + node)[(lane >> 3) & 1] = tot * Wn;
            }
        }
    } else {
    // software pipeline: a node's stencil values are evaluated one iteration before its tile
    // work (so the exp / rsqrt latency overlaps the previous node's loads), from a record
    // loaded two iterations before
    int4 me = make_int4(0, 0, 0, 0), me_n = make_int4(0, 0, 0, 0);
    float Wj = 1.0f, W_n = 1.0f;
    float phv[KV];
    if (ja + half < jb) {
        me = pos[ja + half];
        if (apply_W) Wj = Wv[ja + half];
    }
    ln.values(pos, ja, jb, me, beta, phv);
    if (ja + NPW + half < jb) {
        me_n = pos[ja + NPW + half];
        if (apply_W) W_n = Wv[ja + NPW + half];
    }
    for (int j = ja; j < jb; j += NPW) {
        const int mine = j + half;
        const bool act = (NPW == 1) || mine < jb;
        float phn[KV];
        ln.values(pos, j + NPW, jb, me_n, beta, phn);
        int4 me_nn = make_int4(0, 0, 0, 0);
        float W_nn = 1.0f;
        if (j + 2 * NPW + half < jb) {
            me_nn = pos[j + 2 * NPW + half];
            if (apply_W) W_nn = Wv[j + 2 * NPW + half];
        }
        float k0[L];
#pragma unroll
        for (int q = 0; q < L; q++) k0[q] = (D == 3) ? shfl_slot<KV>(phv, half * DW + q) : 1.0f;
        const int obase = origin_index<G_, D>(me.x & 255, (me.x >> 8) & 255, (me.x >> 16) & 255);
        float accr = 0.0f, acci = 0.0f;
#pragma unroll
        for (int ps = 0; ps < PASSES; ps++) {
            const float kab = shfl_slot<KV>(phv, ln.sa[ps]) * shfl_slot<KV>(phv, ln.sb[ps]);
            if (act && ln.coff[ps] >= 0) {
                const float *pr = tr + obase + ln.coff[ps], *pi = ti + obase + ln.coff[ps];
                float sr = 0.0f, si = 0.0f;
#pragma unroll
                for (int q0 = 0; q0 < L; q0++) {
                    sr = fmaf(k0[q0], pr[q0 * PLANE], sr);
                    si = fmaf(k0[q0], pi[q0 * PLANE], si);
                }
                accr = fmaf(kab, sr, accr);
                acci = fmaf(kab, si, acci);
            }
        }
#pragma unroll
        for (int off = LPN / 2; off > 0; off >>= 1) {  // within each node's lanes
            accr += __shfl_xor_sync(0xffffffffu, accr, off);
            acci += __shfl_xor_sync(0xffffffffu, acci, off);
        }
        if (hl == 0 && act) {
            if constexpr (EN) eacc.add(Wj * (accr * accr + acci * acci), 1.0f);  // W_j |rho_hat_j|^2
            else c_out[mine] = make_float2(accr * Wj, acci * Wj);
        }
        me = me_n;
        me_n = me_nn;
        Wj = W_n;
        W_n = W_nn;
#pragma unroll
        for (int v = 0; v < KV; v++) phv[v] = phn[v];
    }
    }
    if constexpr (EN) {  // energy-only mode: one compensated partial per CTA
        __syncthreads();
        const double2 tot = energy_block_sum(eacc, reinterpret_cast<double *>(smem_raw));
        if (threadIdx.x == 0) epart[blockIdx.x] = tot;
    }
}

// Device-side waits give up after this many polls (each try_wait may also suspend the thread
// for a while); the kernel then sets bit 0 of the plan's status word and returns.
static constexpr long long WAIT_POLLS = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// true when the mbarrier's phase `parity` has completed
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
    for (long long i = 0; i < WAIT_POLLS; i++)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

// Stages the bin's tile of G as 8-byte complex cells, rows of T2 cells (the layout of the TMA
// box), by plain loads: tiles that wrap around the periodic grid or reach into the mirrored
// half (read as conj(G[-l])).
template <typename G_>
__device__ __forceinline__ void stage_tile_cx(const float2 *__restrict__ G, int4 bo, int n, float2 *tile) {
    constexpr int RP = G_::T1 * G_::T2, NC = G_::T0 * RP;
    const bool inside = bo.x >= 0 && bo.x + G_::T0 - 1 <= n / 2;
    for (int cell = threadIdx.x; cell < NC; cell += blockDim.x) {
        const int a0 = cell / RP, rem = cell - a0 * RP, a1 = rem / G_::T2, a2 = rem - a1 * G_::T2;
        tile[cell] = inside ? G[((int64_t)(bo.x + a0) * n + wrap1(bo.y + a1, n)) * n + wrap1(bo.z + a2, n)]
                            : fetch_half<float, 3>(G, n, bo.x + a0, bo.y + a1, bo.z + a2);
    }
}

// FP32 3D interpolation with a lane per node.  The plan orders each bin's nodes in half-groups
// of at most 16 whose stencil origins are equal or fall in different shared-memory bank pairs;
// a warp takes two half-groups, one per half-warp, and its lanes, reading the same stencil
// offset from their own origins, are served without bank conflicts (8-byte loads are served
// per half-warp; equal origins are broadcasts).  Each lane evaluates its node's 3w stencil
// values itself and sums its w^3 cells in registers: no value exchange between lanes and no
// reduction.  The tile (8-byte complex cells, the layout of a TMA box) is loaded by one TMA
// copy when it lies in the stored half without wrapping, else by plain loads.
template <int W>
__device__ __forceinline__ void es_phi_axis(float u, float beta, float (&f)[W]) {
#pragma unroll
    for (int q = 0; q < W; q++) {
        const float vc = ((float)q + 1.0f - 0.5f * (float)W) * (2.0f / (float)W);
        // the first cell reaches |z| = 1 exactly when u = 1 (see F32Lane::values)
        f[q] = (q == 0 && u >= 1.0f) ? 0.0f : es_phi_f32(fmaf(-u, 2.0f / (float)W, vc), beta);
    }
}

// The same w values from the plan's polynomials (NodeDesc::phc, w >= 7): Horner in t = 2u - 1 by
// fused multiply-adds, the coefficients uniform across the warp (kernel-parameter operands).
template <int W>
__device__ __forceinline__ void es_phi_axis_poly(float u, const NodeDesc &nd, float (&f)[W]) {
    constexpr int D = ph_degree(W);
    const float t = fmaf(2.0f, u, -1.0f);
#pragma unroll
    for (int q = 0; q < W; q++) {
        float acc = nd.phc[q * PH_NC + D];
#pragma unroll
        for (int k = D - 1; k >= 0; k--) acc = fmaf(acc, t, nd.phc[q * PH_NC + k]);
        f[q] = (q == 0 && u >= 1.0f) ? 0.0f : acc;  // the edge rule of es_phi_axis
    }
}

template <int W, int BS, bool EN>
__global__ void __launch_bounds__(SUB_THREADS) interp_grp_kernel(NodeDesc nd, const __grid_constant__ CUtensorMap tmap,
                                                                const float2 *__restrict__ G,
                                                                float2 *__restrict__ c_out, int apply_W,
                                                                double2 *__restrict__ epart) {
    pdl_wait();  // (launched by launch_pdl)
    pdl_trigger();
    using G_ = Geo<float, 3, W, BS>;
    constexpr int T0 = G_::T0, T1 = G_::T1, T2 = G_::T2, RP = T1 * T2, NW = SUB_THREADS / 32;
    constexpr unsigned TILE_BYTES = (unsigned)(T0 * RP) * 8u;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the TMA destination must be 128-byte aligned: the launcher adds 128 bytes of room
    float2 *tile = reinterpret_cast<float2 *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    __shared__ __align__(8) unsigned long long mbar;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int4 gs = nd.gsubs[blockIdx.x];
    const int4 bo = nd.bins[gs.z];
    const int n = nd.n;

    // one TMA copy of the box (x0, y0, z0) when the tile sits in the stored half without wrapping:
    // along y and x its cells are bo + a or, for a bin at negative frequencies, n + bo + a
    const bool wrap_y = bo.y < 0 && bo.y + T1 > 0, wrap_x = bo.z < 0 && bo.z + T2 > 0;
    const bool tma = nd.tmap && bo.x >= 0 && bo.x + T0 - 1 <= n / 2 && !wrap_y && !wrap_x &&
                     bo.y + T1 <= n && bo.z + T2 <= n && bo.y >= -n && bo.z >= -n;
    if (tma) {
        const uint32_t mb = smem_u32(&mbar);
        if (threadIdx.x == 0) {
            const int x0 = bo.z < 0 ? bo.z + n : bo.z, y0 = bo.y < 0 ? bo.y + n : bo.y, z0 = bo.x;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(TILE_BYTES)
                         : "memory");
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
                "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(tile)),
                "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(x0), "r"(y0), "r"(z0), "r"(mb)
                : "memory");
        }
        __syncthreads();  // the mbarrier is initialised before anyone polls it
        const bool ok = mbar_wait_bounded(mb, 0);
        if (__syncthreads_or(!ok)) {
            // the copy did not arrive in time (the whole CTA agrees): report, give the copy a
            // second bounded wait to land, and return without reading the tile
            if (threadIdx.x == 0) {
                if (nd.status) atomicOr(nd.status, 1);
                (void)mbar_wait_bounded(mb, 0);
            }
            return;
        }
    } else {
        stage_tile_cx<G_>(G, bo, n, tile);
        __syncthreads();
    }

    const float beta = (float)nd.beta;
    const float *__restrict__ Wv = reinterpret_cast<const float *>(nd.W);
    EAcc<float> eacc;
    const int half = lane >> 4, hl = lane & 15;
    // each lane's next record and weight are loaded one half-group pair ahead, and the
    // half-group bounds that locate them two pairs ahead, so that no record load waits on the
    // load of its own bounds
    const int pend = gs.x + gs.y;
    int pr = gs.x + wid;
    int first = 0, cnt = 0, first_n = 0, cnt_n = 0;
    int4 r_n = make_int4(0, 0, 0, 0);
    float W_n = 1.0f;
    if (pr < pend) {
        first = nd.grp[2 * pr + half];
        cnt = nd.grp[2 * pr + half + 1] - first;
        if (hl < cnt) {
            r_n = nd.pos[first + hl];
            if (apply_W) W_n = Wv[first + hl];
        }
    }
    if (pr + NW < pend) {
        first_n = nd.grp[2 * (pr + NW) + half];
        cnt_n = nd.grp[2 * (pr + NW) + half + 1] - first_n;
    }
    for (; pr < pend; pr += NW) {
        const int4 r = r_n;
        const float Wj = W_n;
        const int node = first + hl;
        const bool mine = hl < cnt;
        if (hl < cnt_n) {  // (cnt_n = 0 past the end)
            r_n = nd.pos[first_n + hl];
            if (apply_W) W_n = Wv[first_n + hl];
        }
        first = first_n;
        cnt = cnt_n;
        if (pr + 2 * NW < pend) {
            first_n = nd.grp[2 * (pr + 2 * NW) + half];
            cnt_n = nd.grp[2 * (pr + 2 * NW) + half + 1] - first_n;
        } else {
            cnt_n = 0;
        }
        if (mine) {
            float fz[W], fy[W], fx[W];
            if (W >= 7 && nd.phpoly) {  // (uniform)
                es_phi_axis_poly<W>(__int_as_float(r.y), nd, fz);
                es_phi_axis_poly<W>(__int_as_float(r.z), nd, fy);
                es_phi_axis_poly<W>(__int_as_float(r.w), nd, fx);
            } else {
                es_phi_axis<W>(__int_as_float(r.y), beta, fz);
                es_phi_axis<W>(__int_as_float(r.z), beta, fy);
                es_phi_axis<W>(__int_as_float(r.w), beta, fx);
            }
            const float2 *pt = tile + ((r.x & 255) * T1 + ((r.x >> 8) & 255)) * T2 + ((r.x >> 16) & 255);
            float ar = 0.0f, ai = 0.0f;
#pragma unroll(W <= 8 ? W : 1)
            for (int qa = 0; qa < W; qa++) {
                float br = 0.0f, bi = 0.0f;
#pragma unroll
                for (int qb = 0; qb < W; qb++) {
                    float sr = 0.0f, si = 0.0f;
#pragma unroll
                    for (int q0 = 0; q0 < W; q0++) {
                        const float2 g = pt[q0 * RP + qa * T2 + qb];
                        sr = fmaf(fz[q0], g.x, sr);
                        si = fmaf(fz[q0], g.y, si);
                    }
                    br = fmaf(fx[qb], sr, br);
                    bi = fmaf(fx[qb], si, bi);
                }
                ar = fmaf(fy[qa], br, ar);
                ai = fmaf(fy[qa], bi, ai);
            }
            if constexpr (EN) eacc.add(Wj * (ar * ar + ai * ai), 1.0f);  // W_j |rho_hat_j|^2
            else c_out[node] = make_float2(ar * Wj, ai * Wj);
        }
    }
    if constexpr (EN) {  // energy-only mode: one compensated partial per CTA
        __syncthreads();
        const double2 tot = energy_block_sum(eacc, reinterpret_cast<double *>(smem_raw));
        if (threadIdx.x == 0) epart[blockIdx.x] = tot;
    }
}

// FP32 spreading.  In 3D each lane forms its column's weight w = c_j phi_1 phi_2 S once per pass
// and a cell's contribution round(w phi_0(q)) by one fused multiply-add (fmaq): half a
// fixed-point unit of rounding, one rounding of the exact product, and no float-to-integer
// conversion per cell.  fmaq needs |w phi_0| <= 2^22, while S only bounds the cell sums (S B <=
// 2^29): a node with S |Re c_j| or S |Im c_j| above 2^22 (one carrying more than about 1/128 of
// its subproblem's sum B) takes the rounded product and a conversion instead (the choice is
// per node, so the same for every lane of its warp: phi <= 1 bounds every column by S |c_j|).
// Lowering S instead, so that every node fits fmaq's range, measured faster (0.94 vs 0.97 ms
// at 256^3) but coarsened the small nodes of dominated subproblems: 3-5x the FP32 error on a
// dipole case.
template <int D, int W, int BS>
__global__ void __launch_bounds__(SUB_THREADS, (Geo<float, D, W, BS>::SPREAD_MINB)) spread_f32_kernel(NodeDesc nd, const float2 *__restrict__ c_in,
                                                                float2 *__restrict__ H) {
    pdl_wait();  // (launched by launch_pdl)
    pdl_trigger();
    using G_ = Geo<float, D, W, BS>;
    using LN = F32Lane<D, W, BS>;
    using F = FixAcc<float>;
    constexpr int PASSES = G_::PASSES, L = (D == 3) ? W : 1, PLANE = G_::PLANE;
    constexpr int LPN = G_::LPN, NPW = G_::NPW, KV = LN::KV, DW = D * W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int *tr = reinterpret_cast<int *>(smem_raw);
    int *ti = tr + G_::NCELL;
    __shared__ float red[2 * (SUB_THREADS / 32)];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int4 sb = nd.subs[blockIdx.x];
    const int4 bo = nd.bins[sb.z];
    LN ln;
    ln.init(nd.pair_order, lane);

    const int ex = spread_scale<float, int, G_::NCELL, F::E, F::MAXEXP>(c_in, sb, tr, ti, red, H);
    if (ex == INT_MIN) return;
    const float S = ldexpf(1.0f, ex);

    int ja, jb;
    warp_chunk(sb, wid, ja, jb);
    const int half = lane / LPN;
    const int4 *__restrict__ pos = nd.pos;
    const float beta = (float)nd.beta;
    if constexpr (LPN == 32 && D == 3) {
        // Two nodes per iteration, as in the interpolation; when they share a stencil origin
        // their two contributions to a cell are added (exactly, in integers) before one shared
        // atomic, so that pair costs the atomics of one node.
        int4 rA_n = make_int4(0, 0, 0, 0), rB_n = make_int4(0, 0, 0, 0);
        float2 cA_n = make_float2(0.0f, 0.0f), cB_n = make_float2(0.0f, 0.0f);
        if (ja < jb) {
            rA_n = pos[ja];
            cA_n = c_in[ja];
        }
        if (ja + 1 < jb) {
            rB_n = pos[ja + 1];
            cB_n = c_in[ja + 1];
        }
        for (int j = ja; j < jb; j += 2) {
            const bool hasB = j + 1 < jb;
            const int4 rA = rA_n, rB = rB_n;
            const float2 cA = cA_n, cB = cB_n;
            if (j + 2 < jb) {
                rA_n = pos[j + 2];
                cA_n = c_in[j + 2];
            }
            if (j + 3 < jb) {
                rB_n = pos[j + 3];
                cB_n = c_in[j + 3];
            }
            float phA[KV], phB[KV];
            ln.values(pos, j, jb, rA, beta, phA);
            ln.values(pos, j + 1, jb, rB, beta, phB);
            float kA[L], kB[L];
#pragma unroll
            for (int q = 0; q < L; q++) {
                kA[q] = shfl_slot<KV>(phA, q);
                kB[q] = shfl_slot<KV>(phB, q);
            }
            const int oA = origin_index<G_, D>(rA.x & 255, (rA.x >> 8) & 255, (rA.x >> 16) & 255);
            const int oB = origin_index<G_, D>(rB.x & 255, (rB.x >> 8) & 255, (rB.x >> 16) & 255);
            const bool same = hasB && rA.x == rB.x;  // the same for every lane
            const float sAr = cA.x * S, sAi = cA.y * S, sBr = cB.x * S, sBi = cB.y * S;
            const bool fast = fmaxf(fmaxf(fabsf(sAr), fabsf(sAi)), fmaxf(fabsf(sBr), fabsf(sBi))) <= FMAQ_MAX;
#pragma unroll
            for (int ps = 0; ps < PASSES; ps++) {
                const float kabA = shfl_slot<KV>(phA, ln.sa[ps]) * shfl_slot<KV>(phA, ln.sb[ps]);
                const float kabB = shfl_slot<KV>(phB, ln.sa[ps]) * shfl_slot<KV>(phB, ln.sb[ps]);
                if (ln.coff[ps] >= 0) {
                    const float wAr = sAr * kabA, wAi = sAi * kabA, wBr = sBr * kabB, wBi = sBi * kabB;
                    int *prA = tr + oA + ln.coff[ps], *piA = ti + oA + ln.coff[ps];
                    int *prB = tr + oB + ln.coff[ps], *piB = ti + oB + ln.coff[ps];
                    // a shared origin: the two contributions are added before one atomic (|A + B|
                    // < 2^30, as each is below S B <= 2^29)
                    if (fast) {
                        if (same) {
                            add_column2<true, L, PLANE>(prA, piA, wAr, wAi, kA, wBr, wBi, kB);
                        } else {
                            add_column<true, L, PLANE>(prA, piA, wAr, wAi, kA);
                            if (hasB) add_column<true, L, PLANE>(prB, piB, wBr, wBi, kB);
                        }
                    } else {
                        if (same) {
                            add_column2<false, L, PLANE>(prA, piA, wAr, wAi, kA, wBr, wBi, kB);
                        } else {
                            add_column<false, L, PLANE>(prA, piA, wAr, wAi, kA);
                            if (hasB) add_column<false, L, PLANE>(prB, piB, wBr, wBi, kB);
                        }
                    }
                }
            }
        }
        __syncthreads();
        flush_tile<float, G_, D, int>(tr, ti, bo, nd, ex, H);
        return;
    }
    // software pipeline as in the interpolation: stencil values one iteration ahead, records
    // and c two iterations ahead
    int4 me = make_int4(0, 0, 0, 0), me_n = make_int4(0, 0, 0, 0);
    float2 c = make_float2(0.0f, 0.0f), c_n = make_float2(0.0f, 0.0f);
    float phv[KV];
    if (ja + half < jb) {
        me = pos[ja + half];
        c = c_in[ja + half];
    }
    ln.values(pos, ja, jb, me, beta, phv);
    if (ja + NPW + half < jb) {
        me_n = pos[ja + NPW + half];
        c_n = c_in[ja + NPW + half];
    }
    for (int j = ja; j < jb; j += NPW) {
        const bool act = (NPW == 1) || j + half < jb;
        float phn[KV];
        ln.values(pos, j + NPW, jb, me_n, beta, phn);
        int4 me_nn = make_int4(0, 0, 0, 0);
        float2 c_nn = make_float2(0.0f, 0.0f);
        if (j + 2 * NPW + half < jb) {
            me_nn = pos[j + 2 * NPW + half];
            c_nn = c_in[j + 2 * NPW + half];
        }
        float k0[L];
        if constexpr (D == 3) {
#pragma unroll
            for (int q = 0; q < L; q++) k0[q] = shfl_slot<KV>(phv, half * DW + q);
        }
        const float csr = c.x * S, csi = c.y * S;
        const bool fast = fmaxf(fabsf(csr), fabsf(csi)) <= FMAQ_MAX;  // the same for the node's lanes
        const int obase = origin_index<G_, D>(me.x & 255, (me.x >> 8) & 255, (me.x >> 16) & 255);
#pragma unroll
        for (int ps = 0; ps < PASSES; ps++) {
            const float kab = shfl_slot<KV>(phv, ln.sa[ps]) * shfl_slot<KV>(phv, ln.sb[ps]);
            if (act && ln.coff[ps] >= 0) {
                int *pr = tr + obase + ln.coff[ps], *pi = ti + obase + ln.coff[ps];
                if constexpr (D == 3) {
                    const float cwr = csr * kab, cwi = csi * kab;
                    if (fast)
                        add_column<true, L, PLANE>(pr, pi, cwr, cwi, k0);
                    else
                        add_column<false, L, PLANE>(pr, pi, cwr, cwi, k0);
                } else {
                    F::add(pr, __float2int_rn(csr * kab));
                    F::add(pi, __float2int_rn(csi * kab));
                }
            }
        }
        me = me_n;
        me_n = me_nn;
        c = c_n;
        c_n = c_nn;
#pragma unroll
        for (int v = 0; v < KV; v++) phv[v] = phn[v];
    }
    __syncthreads();
    flush_tile<float, G_, D, int>(tr, ti, bo, nd, ex, H);
}

template <typename T, int D, int W, int BS>
static cudaError_t launch_interp_w(const NodeDesc &nd, const void *G, void *c_out, int apply_W,
                                   double2 *epart, size_t smem, cudaStream_t s) {
    const unsigned grid = (unsigned)nd.nsub;
    if constexpr (sizeof(T) == 4 && D == 3) {  // lane per node over the plan's node groups
        if (!nd.grp) return cudaErrorInvalidValue;
        const unsigned ggrid = (unsigned)nd.ngsub;
        if (ggrid == 0) return cudaSuccess;
        using G_ = Geo<float, 3, W, BS>;
        // the interleaved tile plus room to align it to 128 bytes (not above the spreading's
        // padded planes of 4-byte cells, which node_smem sizes)
        const size_t tsm = (size_t)G_::T0 * G_::T1 * G_::T2 * 8 + 128;
        const size_t gsm = tsm > smem ? tsm : smem;
        CUtensorMap tm;
        if (nd.tmap) tm = *nd.tmap;
        else std::memset(&tm, 0, sizeof tm);
        if (epart) {
            cudaError_t e = cudaFuncSetAttribute(interp_grp_kernel<W, BS, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
            if (e != cudaSuccess) return e;
            e = launch_pdl(interp_grp_kernel<W, BS, true>, dim3(ggrid), dim3(SUB_THREADS), gsm, s, nd, tm,
                           (const float2 *)G, (float2 *)c_out, apply_W, epart);
            if (e != cudaSuccess) return e;
        } else {
            cudaError_t e = cudaFuncSetAttribute(interp_grp_kernel<W, BS, false>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
            if (e != cudaSuccess) return e;
            e = launch_pdl(interp_grp_kernel<W, BS, false>, dim3(ggrid), dim3(SUB_THREADS), gsm, s, nd, tm,
                           (const float2 *)G, (float2 *)c_out, apply_W, (double2 *)nullptr);
            if (e != cudaSuccess) return e;
        }
    } else if constexpr (sizeof(T) == 4) {
        if (epart) {
            cudaError_t e = cudaFuncSetAttribute(interp_f32_kernel<D, W, BS, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            e = launch_pdl(interp_f32_kernel<D, W, BS, true>, dim3(grid), dim3(SUB_THREADS), smem, s, nd,
                           (const float2 *)G, (float2 *)c_out, apply_W, epart);
            if (e != cudaSuccess) return e;
        } else {
            cudaError_t e = cudaFuncSetAttribute(interp_f32_kernel<D, W, BS, false>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            e = launch_pdl(interp_f32_kernel<D, W, BS, false>, dim3(grid), dim3(SUB_THREADS), smem, s, nd,
                           (const float2 *)G, (float2 *)c_out, apply_W, (double2 *)nullptr);
            if (e != cudaSuccess) return e;
        }
    } else {
        if (epart) {
            cudaError_t e = cudaFuncSetAttribute(interp_sub_kernel<T, D, W, BS, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            e = launch_pdl(interp_sub_kernel<T, D, W, BS, true>, dim3(grid), dim3(SUB_THREADS), smem, s, nd,
                           (const cx_t<T> *)G, (cx_t<T> *)c_out, apply_W, epart);
            if (e != cudaSuccess) return e;
        } else {
            cudaError_t e = cudaFuncSetAttribute(interp_sub_kernel<T, D, W, BS, false>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            e = launch_pdl(interp_sub_kernel<T, D, W, BS, false>, dim3(grid), dim3(SUB_THREADS), smem, s, nd,
                           (const cx_t<T> *)G, (cx_t<T> *)c_out, apply_W, (double2 *)nullptr);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

template <typename T, int D, int W, int BS>
static cudaError_t launch_spread_w(const NodeDesc &nd, const void *c_in, void *H, size_t smem,
                                   cudaStream_t s) {
    const unsigned grid = (unsigned)nd.nsub;
    if constexpr (sizeof(T) == 4) {
        cudaError_t e = cudaFuncSetAttribute(spread_f32_kernel<D, W, BS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = launch_pdl(spread_f32_kernel<D, W, BS>, dim3(grid), dim3(SUB_THREADS), smem, s, nd,
                       (const float2 *)c_in, (float2 *)H);
        if (e != cudaSuccess) return e;
    } else {
        cudaError_t e = cudaFuncSetAttribute(spread_sub_kernel<T, D, W, BS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = launch_pdl(spread_sub_kernel<T, D, W, BS>, dim3(grid), dim3(SUB_THREADS), smem, s, nd,
                       (const cx_t<T> *)c_in, (cx_t<T> *)H);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// Adds the FP64 tiles of the crowded bins into the extended spread grid (one CTA per tile).
template <typename T, int D>
__global__ void __launch_bounds__(SUB_THREADS) crowd_merge_kernel(NodeDesc nd, cx_t<T> *__restrict__ H) {
    pdl_wait();  // (launched by launch_pdl)
    pdl_trigger();
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
    const cudaError_t e = launch_pdl(crowd_merge_kernel<T, D>, dim3((unsigned)nd.ncrowd), dim3(SUB_THREADS),
                                     0, s, nd, (cx_t<T> *)H);
    return e != cudaSuccess ? e : cudaGetLastError();
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

template <typename T, int D, int BS>
cudaError_t launch_interp_bs(const NodeDesc &nd, const void *G, void *c_out, int apply_W,
                             double2 *epart, cudaStream_t s) {
    if (nd.nsub == 0) return cudaSuccess;
    const size_t sm = node_smem(nd, sizeof(T) == 4 ? NLINT_FP32 : NLINT_FP64);
    if (sm > NODE_SMEM_MAX) return cudaErrorInvalidValue;
#define NLINT_CALL_I(WW) launch_interp_w<T, D, WW, BS>(nd, G, c_out, apply_W, epart, sm, s)
    NLINT_W_SWITCH(NLINT_CALL_I)
#undef NLINT_CALL_I
}

template <typename T, int D, int BS>
cudaError_t launch_spread_bs(const NodeDesc &nd, const void *c_in, void *H, cudaStream_t s) {
    if (nd.nsub == 0) return cudaSuccess;
    const size_t sm = node_smem(nd, sizeof(T) == 4 ? NLINT_FP32 : NLINT_FP64);
    if (sm > NODE_SMEM_MAX) return cudaErrorInvalidValue;
#define NLINT_CALL_S(WW) launch_spread_w<T, D, WW, BS>(nd, c_in, H, sm, s)
    NLINT_W_SWITCH(NLINT_CALL_S)
#undef NLINT_CALL_S
}

// One translation unit per (precision, dimension, bin shape), so the width-specialised
// kernels compile in parallel.
#define NLINT_NODE_KERNELS_INSTANTIATE(T, D, BS)                                                \
    template cudaError_t launch_interp_bs<T, D, BS>(const NodeDesc &, const void *, void *, int, \
                                                    double2 *, cudaStream_t);                   \
    template cudaError_t launch_spread_bs<T, D, BS>(const NodeDesc &, const void *, void *,      \
                                                    cudaStream_t);
#define NLINT_CROWD_MERGE_INSTANTIATE(T, D) \
    template cudaError_t launch_crowd_merge_d<T, D>(const NodeDesc &, void *, cudaStream_t);

}  // namespace nlint
