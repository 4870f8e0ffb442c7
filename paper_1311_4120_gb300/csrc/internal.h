// Internal declarations shared by the host plan code and the kernel launchers.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "nlint.h"

namespace nlint {

// Sets the calling thread's nlint_last_error message and returns `code`.
int report_error(int code, const char *msg);

// ---------------------------------------------------------------------------- FFT passes
// One pass transforms every line along one axis of a 2D/3D array.  A "column" pass works
// on an axis that is not contiguous (the batch index is contiguous); a "row" pass works on
// the contiguous axis.
enum InKind {
    IN_REAL_MODES = 0,   // N reals at centred mode positions, times the deconvolution product
    IN_CPLX_MODES = 1,   // N complex at centred mode positions
    IN_CPLX_FULL = 2,    // n complex
    IN_CPLX_HERM = 3,    // n/2+1 complex of a Hermitian line (rest by conjugate symmetry)
    IN_CPLX_FOLD = 4,    // row pass only: n complex plus the conjugated mirror row (fold)
    IN_CPLX_WIN = 6      // the 2 win + 1 window entries (FFT index e <= win or e >= n - win),
                         // stored compactly (e, then e - n + 2 win + 1); zero elsewhere
};
enum OutKind {
    OUT_CPLX_FULL = 0,   // n complex
    OUT_CPLX_HALF = 1,   // first n/2+1 complex
    OUT_CPLX_MODES = 2,  // N complex at centred mode positions
    OUT_REAL_MODES = 3,  // N reals (real part) times the deconvolution product, + energy
    OUT_CPLX_WIN = 4     // the 2 win + 1 window entries, compact (as IN_CPLX_WIN)
};

struct PassDesc {
    int n;               // FFT length
    int nrad;
    int rad[12];         // radix sequence (8, 4, 2, 3)
    int sign;            // -1 forward, +1 backward
    int N;               // number of modes per axis
    int in_kind, out_kind;
    int dim;             // d, for the deconvolution product over the batch index
    int64_t I;           // batch length along the contiguous index (column pass) / rows (row pass)
    int64_t n_outer;     // outer count (column pass)
    int64_t in_so, in_sa;    // element strides: outer, axis (column pass); row stride (row pass)
    int64_t out_so, out_sa;
    int B, TPC, LD;      // columns (or rows) per CTA, threads per column, smem leading dim
    // fold (row pass over the extended spread grid): see the row-pass kernel
    int fold_pad;        // pad planes below/above the stored half of the slowest axis
    int64_t fold_plane;  // elements per plane of the slowest axis (rows per plane * n)
    int64_t fold_rows_per_plane;
    const void *fac;     // deconvolution factors, length N (plan precision)
    const void *mult;    // conv (mode 5): real multiplier, one n-entry row per line
    const void *rho;     // energy: density (OUT_REAL_MODES)
    double2 *partials;   // energy: one compensated partial per CTA (OUT_REAL_MODES)
    int accum;           // OUT_REAL_MODES: add to the output instead of overwriting it
    // frequency window (0 = none): only FFT indices e <= win or e >= n - win are nonzero or
    // needed.  IN_CPLX_HERM reads zero outside it, OUT_CPLX_HALF writes e <= win only,
    // OUT_CPLX_FULL writes the window entries only (at their full-line index).
    int win;
    // 3D row passes over a window (win_rows = 2 win + 1): row q is plane q / win_rows and
    // window row q % win_rows, i.e. full-grid row c (c <= win) or n - (win_rows - c); the fold
    // reads, and an OUT_CPLX_FULL pass writes, that full-grid row
    int win_rows;
    // row pass that convolves each line (mode 5): forward FFT of the N input modes, times the
    // real n-entry row `mult` + q n, inverse FFT, N output modes
    int conv;
    // dual column pass (modes 6, 7) of two transforms that share the density and u: I_1 with the
    // unit factors `fac` and I_2 with the deconvolution factors `fac2` over the window `win`.
    // Forward (IN_REAL_MODES -> OUT_CPLX_HALF): I_1's half to the output, I_2's window planes
    // (e <= win, same strides) to `out2`.  Inverse (IN_CPLX_HERM -> OUT_REAL_MODES): I_1's half
    // from the input, I_2's window planes from `in2`, u = the sum of the two (+ energy).
    int dual;
    const void *fac2;
    const void *in2;
    void *out2;
    // ball window of the full row passes along x (0 = none): every fine cell a node's stencil
    // touches has s0^2 + s1^2 + s2^2 <= ball2 (signed FFT indices), so the forward row pass
    // (mode 1) writes, and the fold pass (mode 2) reads, only the entries of each row inside that
    // ball (rows outside it: nothing written; the fold pass writes their zero transform).  For
    // the convolution pass (mode 5) every multiplier row with s0^2 + s1^2 > ball2 is zero, so
    // those rows write zeros without transforming
    int64_t ball2;
    int sched;           // schedule variant of this pass (0 or 1), set by config_pass
};

void make_radix(int n, PassDesc &p);
bool fft_size_supported(int n);   // n = 2^a or 3*2^a, 16 <= n <= 2048
int fft_next_size(int64_t m);     // smallest supported size >= m, or -1
int64_t pass_blocks(const PassDesc &p, bool row);
int pass_threads(const PassDesc &p);
size_t pass_smem(const PassDesc &p, int prec);
// CTA geometry of a pass; `sched` is the plan's schedule mask (nlint_params.fft_sched: bit 0
// column passes, 1 row passes, 2 the fold pass, 3 the packed real-data passes; FP32 only)
void config_pass(PassDesc &p, int prec, bool row, unsigned sched = 0);
bool pass_fits(const PassDesc &p);

// pass mode 0: column pass; 1: row pass; 2: row pass reading the fold input;
// 3: column pass real -> Hermitian half, two lines per FFT; 4: Hermitian half -> real, two lines;
// 5: row pass forward FFT, multiply, inverse FFT; 6, 7: dual column passes (forward, inverse)
int pass_mode(const PassDesc &p, bool row);
// Launch of a pass of mode MODE with schedule V (see fft_kernels.cuh); launch_pass_mode picks V
// from the descriptor (p.sched, FP32 modes 0-4 only).
template <typename T, int MODE, int V>
cudaError_t launch_pass_mode_v(const PassDesc &p, const void *in, void *out, const void *tw,
                               cudaStream_t s);
template <typename T, int MODE>
cudaError_t launch_pass_mode(const PassDesc &p, const void *in, void *out, const void *tw,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_colpass(const PassDesc &p, const void *in, void *out, const void *tw,
                           cudaStream_t s);
template <typename T>
cudaError_t launch_rowpass(const PassDesc &p, const void *in, void *out, const void *tw,
                           cudaStream_t s);

// ---------------------------------------------------------------------------- NUFFT kernels
// The half node set, sorted by bin.  A bin is a box of B[0] x B[1] (x B[2]) stencil-origin
// cells; the union of its nodes' stencils lies in a tile of T[a] = B[a] + w - 1 cells per axis
// starting at the bin's origin.  A subproblem is a run of at most a few hundred nodes of one
// bin and is processed by one CTA on a shared-memory copy of the tile.  Axis 0 is the half
// (slowest) axis; in 2D only axes 0 and 1 are used.
static constexpr int NODE_MAXW = 16;     // widest stencil
// Stencil-value polynomials of the FP32 3D interpolation: degree 8 at w = 7, 7 above (the fits
// reach about 1e-7 absolute in FP32 there; below w = 7 the function's square-root edge at
// |z| = 1 carries exp(-beta) >= 1e-6 and the formula is kept)
constexpr int PH_NC = 9;
__host__ __device__ constexpr int ph_degree(int w) { return w == 7 ? 8 : 7; }

struct NodeDesc {
    int d;
    int64_t M;           // number of nodes (half set)
    int n;               // fine grid size per axis
    int w;               // stencil width
    int pad;             // extended planes below/above the half grid (slowest axis)
    double beta;         // ES kernel shape parameter
    int bin_shape;       // bin shape (see bin_dim); the kernels are compiled per shape
    // FP32 plans: one 16-byte record per node, {r0 | r1 << 8 | r2 << 16, u_0, u_1, u_2}: the
    // first stencil cell per axis relative to the bin origin and, as float bits, the offset
    // u_a = frac_a - (w/2 - 1) in (0, 1] of the node from that cell (frac_a = g_a - first
    // cell); the kernels evaluate the stencil values from u_a.  FP64 plans: rel and ker.
    const int4 *pos;
    const int32_t *rel;  // M: first stencil cell relative to the bin origin, r0 | r1 << 8 | r2 << 16
    const void *ker;     // M x (d w): kernel values phi((q - frac_a)/(w/2)), row per node
    const void *W;       // M, h^d W_j (plan precision), may be NULL (type-2 only)
    int B[3], T[3];      // bin and tile extents per array axis
    int64_t nsub;        // number of subproblems
    const int4 *subs;    // per subproblem {first node, node count, bin, 0}
    // FP32 3D plans: the nodes of each bin are ordered in half-groups of at most 16 whose
    // stencil origins share no shared-memory bank pair unless they are equal (see
    // build_node_groups); the interpolation gives each node of a half-group a lane of its own,
    // two half-groups (one per half-warp) per warp
    int64_t ngsub;       // interpolation subproblems (runs of half-group pairs of one bin)
    const int4 *gsubs;   // per interpolation subproblem {first pair, pair count, bin, 0}
    const int32_t *grp;  // half-group g holds nodes grp[g] .. grp[g + 1] - 1 (bins: even counts)
    // FP32 3D Algorithm 1 plans: a tiled tensor map of the fine grid G (8-byte cells, the
    // stored half: n x n x (n/2 + 1)) from which the interpolation stages its tiles by TMA;
    // NULL: plain loads
    const CUtensorMap *tmap;
    int *status;         // device word: bit 0 set when a bounded wait in a kernel ran out
    const int4 *bins;    // per bin {origin axis 0, axis 1, axis 2, crowd slot or -1}
    int ncrowd;          // crowded bins (FP32 plans): their tiles are summed in FP64
    double2 *crowd;      // ncrowd tiles of complex doubles
    const int32_t *crowd_bin;  // bin of each crowd slot
    const int16_t *pair_order; // per pass and node lane: column (q_a << 8 | q_b) or -1 (spreading)
    const int16_t *pair_order_i;  // the same for the interpolation (8-byte tile cells)
    // FP32 3D interpolation, w >= 7: phi on each of the w stencil cells as a polynomial of degree
    // ph_degree(w) in t = 2 u - 1 (u the node's offset, as above), monomial coefficients
    // phc[q * PH_NC + k] (k = 0 lowest); phpoly = 0: evaluate phi by its formula instead
    int phpoly;
    float phc[NODE_MAXW * PH_NC];
};

// Deals the w*w stencil columns (q_a, q_b) of a node to passes of `lanes` lanes so that,
// within a pass, the tile offsets q_a * row + q_b of each group of `group` lanes (the lanes one
// shared-memory wavefront serves: 32 for 4-byte, 16 for 8-byte elements) fall in distinct
// banks where possible (`banks` = 32 for 4-byte, 16 for 8-byte elements).  Returns
// passes * lanes entries.
std::vector<int16_t> build_pair_order(int w, int row, int banks, int lanes, int group);

// Splits one bin's nodes (indices first .. first + count - 1, sorted by stencil origin; org[i]
// is node i's origin as a tile offset in cells) into groups of at most `lanes` nodes in which
// two nodes have either the same origin or origins whose offsets differ mod `banks` (different
// shared-memory banks, or bank pairs for 8-byte cells).  A lane per node then reads the node's
// stencil (the same offsets from every origin) without bank conflicts.  Greedy: origins with
// the most remaining nodes first, each group taking as many nodes of one origin as fit.
// Appends the bin's new node order to `order` and each group's size to `sizes`.
void build_node_groups(const int32_t *org, int64_t first, int64_t count, int lanes, int banks,
                       std::vector<int64_t> &order, std::vector<int> &sizes);

// Bin shapes (stencil-origin cells per array axis).  3D: 1 = 8 x 8 x 8, 2 = 4 x 8 x 8,
// 3 = 8 x 16 x 16, 4 = 16 x 16 x 16; 2D: 16 x 16 for every shape.  The kernels are compiled
// per shape (FP32 3D: shapes 1, 3, 4; FP64 3D: 1, 2; 2D: 1), so a plan's bins always match the
// tile geometry of its kernels.  A tile is bin + w - 1 cells per axis.
static constexpr int NBIN_SHAPES = 4;
__host__ __device__ constexpr int bin_dim(int d, int bs, int axis) {
    return d == 2 ? (axis < 2 ? 16 : 1)
                  : (bs == 2 ? (axis == 0 ? 4 : 8)
                             : bs == 3 ? (axis == 0 ? 8 : 16) : bs == 4 ? 16 : 8);
}
// Whether kernels are compiled for a (precision, dimension, shape).
__host__ __device__ constexpr bool bin_shape_built(bool fp64, int d, int bs) {
    return d == 2 ? bs == 1 : (fp64 ? (bs == 1 || bs == 2) : (bs == 1 || bs == 3 || bs == 4));
}
// The shape a plan takes when none is requested: FP64 3D 4 x 8 x 8 for w >= 10 (tile within
// 100 KB of shared memory), else 8 x 8 x 8; FP32 3D 8 x 16 x 16.
__host__ __device__ constexpr int default_bin_shape(bool fp64, int d, int w) {
    return d == 2 ? 1 : (fp64 ? (w >= 10 ? 2 : 1) : 3);
}

// Lanes per node in the interpolation / spreading kernels: 16 when the w*w stencil columns
// waste fewer lane slots in passes of 16 than in passes of 32 (w = 4, 6, 10..13, ...), else 32.
__host__ __device__ constexpr int node_lanes(int w) {
    return (w * w + 15) / 16 * 16 < (w * w + 31) / 32 * 32 ? 16 : 32;
}
static constexpr int NODE_THREADS = 256;  // threads per interpolation / spreading CTA

// Shared-memory row pitch of a 3D FP32 tile (cells between consecutive axis-1 rows; at least
// the tile extent bin + w - 1 along axis 2).  A node's lanes read (or add to) its w*w stencil
// columns, at offsets pitch * q_a + q_b, in passes of node_lanes(w) lanes; the smallest pitch
// whose offsets fall at most `passes` times in any of the 32 banks lets every pass hit distinct
// banks (an 8 x 16 x 16 bin at w = 7 has rows of 22 cells, whose offsets miss three banks and
// doubled a third of all shared wavefronts; a pitch of 23 removes that).  FP64 and 2D tiles
// keep the extent.
__host__ __device__ constexpr int tile_pitch(bool fp64, int d, int w, int bs) {
    const int t2 = (d == 3 ? bin_dim(d, bs, 2) : bin_dim(d, bs, 1)) + w - 1;
    if (fp64 || d != 3) return t2;
    const int lanes = node_lanes(w), passes = (w * w + lanes - 1) / lanes;
    for (int p = t2; p < t2 + 9; p++) {
        int cnt[32] = {};
        int mx = 0;
        for (int a = 0; a < w; a++)
            for (int b = 0; b < w; b++) {
                const int r = (p * a + b) % 32;
                cnt[r]++;
                mx = cnt[r] > mx ? cnt[r] : mx;
            }
        if (mx <= passes) return p;
    }
    return t2;
}

int tile_cells(const NodeDesc &nd);
size_t node_smem(const NodeDesc &nd, int prec);
// Dynamic shared memory of the node kernels for a plan geometry (tile planes, plus the FP64
// kernels' per-warp stencil-value tables); must not exceed NODE_SMEM_MAX.
size_t node_smem_for(int prec, int d, int w, int bs);
// (the opt-in limit per CTA, 227 KB, less 1 KB for the kernels' static shared arrays)
static constexpr size_t NODE_SMEM_MAX = 227 * 1024 - 1024;

// c_out[j] = (apply_W ? W_j : 1) rho_hat_j / h^d; with epart != NULL nothing is written to
// c_out and each CTA writes sum_j W_j |rho_hat_j / h^d|^2 over its nodes to epart[cta]
template <typename T>
cudaError_t launch_interp(const NodeDesc &nd, const void *G, void *c_out, int apply_W,
                          cudaStream_t s, double2 *epart = nullptr);
template <typename T>
cudaError_t launch_spread(const NodeDesc &nd, const void *c_in, void *Hext, cudaStream_t s);
template <typename T>
cudaError_t launch_crowd_merge(const NodeDesc &nd, void *Hext, cudaStream_t s);
// per (precision, dimension, bin shape) launchers, one translation unit each (width dispatch
// inside); only the combinations bin_shape_built() names exist
template <typename T, int D, int BS>
cudaError_t launch_interp_bs(const NodeDesc &nd, const void *G, void *c_out, int apply_W,
                             double2 *epart, cudaStream_t s);
template <typename T, int D, int BS>
cudaError_t launch_spread_bs(const NodeDesc &nd, const void *c_in, void *Hext, cudaStream_t s);
template <typename T, int D>
cudaError_t launch_crowd_merge_d(const NodeDesc &nd, void *Hext, cudaStream_t s);

template <typename T>
cudaError_t launch_scatter_canonical(int64_t M, const void *vals, const int32_t *perm,
                                     const int32_t *mirror, double scale, void *out,
                                     cudaStream_t s);
template <typename T>
cudaError_t launch_gather_canonical(int64_t M, const void *c_canon, const int32_t *perm,
                                    const int32_t *mirror, void *c_half, cudaStream_t s);
template <typename T>
cudaError_t launch_energy_partials(int64_t count, const void *u, const void *rho,
                                   double2 *partials, int nblocks, cudaStream_t s);
// E = scale * (compensated sum of the nparts partials), in a fixed order.  The buffer must hold
// nparts + 64 entries: the last 64 are scratch for the two-stage fold.
cudaError_t launch_energy_final(const double2 *partials, int nparts, double scale, double *E,
                                cudaStream_t s);
int energy_final_kernels(int nparts);  // kernels launch_energy_final launches (1 or 2)
// Toeplitz kernel assembly: an N^d block into an n^d array at cell offsets off = (slowest,
// middle, fastest array axis; 2D: slowest, -, fastest)
template <typename T>
cudaError_t launch_place_block(int d, int64_t N, int64_t n, int3 off, const void *u, double scale,
                               void *K, cudaStream_t s);
template <typename T>
cudaError_t launch_extract_real(int64_t cnt, const void *G, double scale, void *khat, cudaStream_t s);

}  // namespace nlint
