// Internal interface between the host side of the library (api.cu) and the
// device kernels (engine.cu, binning.cu).  Not part of the public C ABI.
//
// Data layout of the d-dimensional transform (Sec. 4, steps 2-4):
//   A "work item" is one complex transform.  For a kernel item it carries two
//   real lag kernels packed as k_A + i k_B (both are even, k_{-j} = k_j, so
//   their transforms are real and come back as the real and imaginary parts);
//   for a counts item it carries the grid counts.  Along axis k the input is
//   nonzero only on S_k consecutive dense indices idx (the support
//   |j_k| <= L_k of Eq. 25, or the M_k grid nodes); dense index idx sits at
//   circular position p = (idx - off_k) mod P_k of the zero-padded line.
//   Axes are transformed last to first.  After axes k..d-1 are done the
//   scratch holds [w_{d-1}][w_{d-2}]..[w_k][i_0..i_{k-1}] (the last axis keeps
//   only w_{d-1} in [0, P_{d-1}/2], the other half follows from the
//   symmetry K(-w) = conj(K(w)) of a real input).  The final pass transforms
//   axis 0 and either reduces against the count spectrum (kernel items) or
//   writes |Y|^2 (counts items); the spectrum layout is [q][w_0] with
//   q = flattened (w_{d-1}, .., w_1), w_{d-1} outermost.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kdefft {

constexpr int MAXD = 4;
constexpr int MAXSIG = 3;
constexpr int MAXTERM = 40;
constexpr int MAXST = 14;     // radix stages per axis (P <= 4096)
constexpr int MAXP = 4096;
constexpr int HMAX = 216;     // Hermite table entries: C(D+R, D) for (D,R) = (4,6) is 210

// Recurrence program for the multivariate Hermite polynomials He_alpha(z;
// Lambda), graded order (all |alpha| = 0, then 1, ...).  Entry t > 0:
//   He[t] = z[piv] He[par] - sum_q rc[q] Lambda[piv][rj[q]] He[ridx[q]].
struct HEnt {
    uint16_t par;
    uint8_t piv;
    uint8_t nred;
    uint8_t rj[MAXD];
    uint8_t rc[MAXD];
    uint16_t ridx[MAXD];
};

struct AxisPlan {
    int P;
    int nst;
    int tw_off;                 // offset of exp(-2 pi i t / P), t < P, in the twiddle pool
    unsigned char radix[MAXST];
};

template <typename real>
struct Item {
    int d;
    int kind;                   // 0: kernel pair reduced against a spectrum; 1: counts -> |C|^2
    AxisPlan ax[MAXD];
    int S[MAXD];                // support length per axis
    int off[MAXD];              // position p = (idx - off) mod P
    int R;                      // highest derivative order in the terms
    int nsig;                   // distinct covariances
    double lam[MAXSIG][MAXD * MAXD];   // Sigma^{-1}, row stride MAXD (FP64: the quadratic form is FP64)
    double nrm[MAXSIG];         // (2 pi)^{-d/2} |Sigma|^{-1/2}
    double delta[MAXD];         // bin widths (Eq. 16)
    int nterm[2];
    short tsig[2][MAXTERM];
    short the[2][MAXTERM];
    real tw8[2][MAXTERM];       // weights, sign (-1)^{|alpha|} folded in
    const real* spec;           // kind 0: count spectrum |C|^2, layout [q][w0]
    const real* counts;         // kind 1: counts, row-major over M
    real* spec_out;             // kind 1: output spectrum
    long long scr[2];           // scratch offsets (complex elements)
    int tileF0, ntileF;         // range of final-pass tiles (their partial sums)
    double scale;               // n^-2 / prod P_k
};

// One unit of a pass: item index, then pass-specific fields
//   stage A: a = first line, n = lines
//   mid:     a = outer transformed index wo, b = first inner line o0, n = lines
//   final:   a = first q, n = lines
struct Tile {
    int item;
    int a;
    int b;
    int n;
};

template <typename real>
struct Cpx;
template <>
struct Cpx<float> { using T = float2; };
template <>
struct Cpx<double> { using T = double2; };

// Host-side launchers (engine.cu).  cap: complex elements per ping-pong
// buffer in shared memory; pmax: largest P of the pass (its twiddles are
// staged in shared memory); twpool: device table of all twiddles.
template <typename real>
cudaError_t launch_stage_a(const Item<real>* items, const Tile* tiles, int ntiles, int pmax, int cap,
                           typename Cpx<real>::T* scratch, const typename Cpx<real>::T* twpool, double* partial,
                           int grid, cudaStream_t st);
template <typename real>
cudaError_t launch_mid(const Item<real>* items, const Tile* tiles, int ntiles, int axis, int pmax, int cap,
                       typename Cpx<real>::T* scratch, const typename Cpx<real>::T* twpool, int grid,
                       cudaStream_t st);
template <typename real>
cudaError_t launch_final(const Item<real>* items, const Tile* tiles, int ntiles, int pmax, int cap,
                         typename Cpx<real>::T* scratch, const typename Cpx<real>::T* twpool, double* partial,
                         int grid, cudaStream_t st);
template <typename real>
cudaError_t launch_reduce(const Item<real>* items, int nitems, const double* partial, double* out,
                          cudaStream_t st);

// Work item of the fused 2-D kernel, prepared on the host: the fields its
// inner loops read, with the kernel terms expanded into dense weights
// W[grid][covariance][Hermite index] (sign (-1)^{|alpha|} included); the
// kernel stages it in shared memory.  Size is a multiple of 4 bytes.
constexpr int WDENSE = 15;   // C(2 + 4, 2): d = 2 up to order 4
template <typename real>
struct FusedItem {
    int S0, S1, off0, off1, nsig, pad_;
    double delta0, delta1;
    double lam[MAXSIG][4];   // Sigma^{-1} (FP64: the quadratic form is FP64)
    real laml[MAXSIG][4];    // the same in the working type, for the Hermite recurrence
    real nrm[MAXSIG];
    real W[2][MAXSIG][WDENSE];
    // device search, SCV only: for s = 0 (2H + 2G) and 1 (H + 2G), in
    // lag-index coordinates (x = delta (.) j): the exponent difference
    // x^T (Sigma_s^-1 - (2G)^-1) x = j^T D_s j, entries 00, 01, 11 as FP32
    // leading parts [0..2] and remainders [3..5]; the normaliser ratio
    // rho_s = phi_{Sigma_s}(0) / phi_{2G}(0) [6, 7] and rho_s - 1 [8, 9],
    // each as an FP32 pair
    real xd[2][12];
    AxisPlan a0, a1;
    const real* spec;
    double scale;
};

// d = 2: one thread-block cluster of cs CTAs per item does stage A, the
// final pass and the reduction (out[2 i], out[2 i + 1], scaled).
// gat_elems: complex elements per CTA for the inputs of its axis-0 lines
// (S_0 x columns per CTA); spc_elems: reals for its spectrum rows (columns x
// P_0); cap: per ping-pong buffer.  errflag: set to 1 if a bounded wait on
// the spectrum copy gave up.
// rmax: highest derivative order among the items' terms (<= 4; larger
// orders return cudaErrorNotSupported and the caller uses the multi-pass path).
template <typename real>
cudaError_t launch_fused2d(const FusedItem<real>* items, int nitems, int rmax, int cs, int gat_elems, int spc_elems,
                           int cap, int pmax, const typename Cpx<real>::T* twpool, double* out, int* errflag,
                           cudaStream_t st);

// ---- device-resident bandwidth selection (d = 2, FP32): one cluster per
// start runs the whole quasi-Newton search; see k_select2d in engine.cu.
struct SelSpec {            // one padded-size pair and its count spectrum
    int P0, P1;
    AxisPlan a0, a1;
    const float* spec;
    double scale;           // 1 / (n^2 P_0 P_1)
    double fl_line, fl_fix, by;   // algorithmic work of one evaluation: fl_fix + S_0 fl_line flops, by bytes
};
struct SelStart {           // in: start point; out: end point
    double th[3];           // Cholesky parameters (log R00, R10, log R11)
    double f;
    double flops, bytes;    // out: algorithmic work of this start's evaluations
    int evals, iters, status;   // status: 0 converged / stalled, 1 iteration cap, 2 no valid start
};
struct SelectParams {
    int method;             // 0: LSCV (Eq. 10), 1: SCV (whole kernel in FP32)
    int max_iter;
    int cs;                 // CTAs per cluster
    int nspec;
    int widest;             // LSCV: support from lambda_max(2H) instead of lambda_max(H)
    int M0, M1;
    int Lcap, Lcap1;        // trial points needing a larger support (axis 0, axis 1) are outside the search
    int chunk;              // lines (and columns) per shared-memory batch
    int gat_elems, spc_elems, cap, pmax;   // shared-memory layout (complex / real elements)
    double n, tau;
    double inv_n, inv_n2;   // 1/n, 1/n^2
    float inv_nf;           // 1/n in FP32
    float inv_n2h, inv_n2l; // 1/n^2 as an FP32 pair (h + l)
    float tauf, d0f, d1f;   // tau, delta_0, delta_1 rounded to FP32
    float rd0f, rd1f;       // 1 / d0f, 1 / d1f, correctly rounded (as __frcp_rn)
    float Gf[4];            // G rounded to FP32
    // SCV, each from FP64 on the host: (2G)^-1 (entries 00, 01, 11), its
    // determinant and delta_0^2, delta_0 delta_1, delta_1^2 as FP32 pairs
    // (h, l); (2G)^-1 in lag-index coordinates, delta_a delta_b (2G)^-1_ab,
    // and phi_{2G}(0) rounded to FP32; the lag-index to H-gradient factors
    // 1 / (delta_0^2), 1 / (delta_0 delta_1), 1 / (delta_1^2)
    float l2gh[3], l2gl[3], dl2gh, dl2gl, ddh[3], ddl[3];
    float l2gj[3], n2g, gsc[3];
    double delta0, delta1;
    double G[4];            // SCV pilot, row-major
    const int* ptab0;       // P_0 for support L_0 (index L_0 <= Lcap)
    const int* ptab1;
    const SelSpec* specs;
    int* errflag;
    // lag domain (k_select2d_lag): the FP32 count autocorrelation on the half
    // box [j_1 + A1][j_0], j_0 in [0, A0]; null for the FFT route
    const float* acorr;
    int A0, A1;
    // optional record of the search's own evaluations (null: off): for CTA
    // (start) s, evaluation e < rec_cap goes to rec + (s rec_cap + e) SEL_REC
    double* rec;
    int rec_cap;
};
// fields of one recorded evaluation: start, evaluation index, method, H_00,
// H_01, H_11 (the FP32 values evaluated), L_0, L_1, value, dF/dH_00,
// dF/dH_01 (tied), dF/dH_11
constexpr int SEL_REC = 12;
cudaError_t launch_select2d(const SelectParams& prm, SelStart* starts, int nstarts,
                            const float2* twpool, cudaStream_t st);
// the same search in the lag domain: one CTA per start (prm.acorr set).
// Starts [0, nfirst) search with prm, the rest with prm2; both share the
// autocorrelation box (acorr, A0, A1) of prm.
cudaError_t launch_select2d_lag(const SelectParams& prm, const SelectParams& prm2, int nfirst, SelStart* starts,
                                int nstarts, cudaStream_t st);

cudaError_t upload_hermite_tables(const HEnt* tab, const int* offsets, int total);
// raise the dynamic shared-memory limits (and cluster permissions) of the
// engine's kernels on the current device; once per device, before launches
cudaError_t prepare_kernels();

// ---- lag-domain engine (lag.cu)
// Eq. 25 summed over the lag first: n^-2 sum_i sum_j c_i c_j k(i - j) =
// n^-2 sum_l k_l a_l with the count autocorrelation a_l = sum_i c_i c_{i+l}.
// Both k (even-order Gaussian partials) and a are even, so the sum runs over
// the half box j_0 in [0, L_0], j_k in [-L_k, L_k] (k >= 1) with weight 2 on
// points whose first nonzero coordinate is positive, 1 at j = 0, 0 otherwise.
// The autocorrelation array holds the half box of a larger box A, layout
// [j_{d-1}]..[j_1][j_0] (j_0 innermost, j_k + A_k for k >= 1).
template <typename real>
struct LagItem {
    int d, nsig, R, pad_;
    int L[MAXD];                      // support of this item's kernels
    int A[MAXD];                      // box of the autocorrelation array
    // division of a flat half-box index by the extents L_0 + 1, 2 L_k + 1
    // (axes 0 .. d - 2) as a multiply-high: multiplier and shifts s1 | s2 << 8
    // of Granlund and Montgomery's unsigned division by an invariant integer
    unsigned int qm[MAXD];
    int qs[MAXD];
    real lam[MAXSIG][MAXD * MAXD];    // Sigma^{-1}, row stride MAXD
    real nrm[MAXSIG];                 // (2 pi)^{-d/2} |Sigma|^{-1/2}
    real delta[MAXD];
    const real* acorr;
    int w_off;                        // dense weights [2][nsig][N(d, R)] at wpool + w_off
    int tile0, ntile;                 // this item's tiles (their partial sums)
    double scale;                     // n^-2
};
struct LagTile {
    int item;
    int n;                            // points of the item's half box in this tile
    long long first;                  // first flat index (j_0 fastest)
};
// Number of Hermite entries C(d + R, d) of the compile-time tables, or 0 when
// no lag kernel is instantiated for (d, R, real) (the caller uses the FFT path).
int lag_table_size(int d, int R, bool dbl);
// One launch of the lag kernel over tiles [t0, t0 + ntiles) of a batch (one
// derivative-order class): items, tiles and weights of the batch, partial
// (2 per tile of the batch).
// FP64 lag tiles hold 32 * kLagSlices points, one per thread, in kLagSlices
// warp slices; each slice writes its own partial pair (kLagSlices per tile),
// which k_lag_sum combines in a fixed order.  So a launch may run one slice
// per 32-thread CTA (few tiles: the slow FP64 points spread over the SMs) or
// a whole tile per 256-thread CTA, with the same bits.  FP32 tiles write one
// partial pair each.
constexpr int kLagSlices = 8;
template <typename real>
struct LagJob {
    const LagItem<real>* items;
    const LagTile* tiles;
    int t0, ntiles, grid;
    int block;                        // 256; FP64 also 32, 64 or 128 (slices per CTA = block / 32)
    const real* wpool;
    double* partial;                  // per tile of the batch: 1 pair (FP32) or kLagSlices pairs (FP64)
};
template <typename real>
cudaError_t launch_lag(int d, int R, const LagJob<real>& j, cudaStream_t st);
// An item's tile partials (tile0 indexes the run's whole partial buffer, in
// pairs) and its scale n^-2: the per-item sums of a run, whatever the
// batch's precision.
struct LagSum {
    long long tile0;                  // first partial pair of the item's first tile
    int ntile, nslice;                // tiles; partial pairs per tile (1 or kLagSlices)
    double scale;
};
cudaError_t launch_lag_sum(const LagSum* sums, int nitems, const double* partial, double* out, cudaStream_t st);
// One separable pass of the inverse DFT that turns the FP64 count spectrum
// into the autocorrelation, for one dataset: out[o][jj][i] = sum_{w < W} h(w)
// in[o][w][i] e^{+2 pi i w (jlo + jj) / P}, h(w) = 1, or for the
// half-spectrum axis (half != 0) 1 at w = 0 and w = P/2 and 2 elsewhere.  in:
// real (in_r) or complex (in_c); out: complex (out_c), or the real part times
// `scale` (out_r, and rounded to FP32 into out_r32 when given).  Twiddles
// exp(-2 pi i t / P), t < P, at twpool + tw_off.  blk0: the job's first
// block in a launch over many jobs (set by the launcher).
struct AcorrJob {
    const double* in_r;          // real input (the count spectrum; first pass, I = 1), or
    const double2* in_c;         // complex input of a later pass
    double2* out_c;              // complex output of a pass before the last, or
    double* out_r;               // real part of the last pass (times scale), with
    float* out_r32;              // its FP32 copy
    long long O, I;              // lines O I; element (o, w, i) at (o W + w) I + i
    int W, J, jlo, half;         // W values per line (<= P); lags jlo .. jlo + J - 1; half: weights 2 inside
    int nl;                      // lines per CTA
    AxisPlan ap;                 // the length-P transform (radix stages, twiddle offset)
    double scale;
    long long blk0;
};
// shared memory of an autocorrelation pass: two line buffers and P twiddles
__host__ __device__ constexpr size_t acorr_smem_bytes(int P, int nl) {
    return sizeof(double2) * ((size_t)2 * (size_t)(nl * P + ((nl * P) >> 4) + 1) + (size_t)P);
}
// All jobs' passes of one level in one launch (one CTA per nl lines).
// acorr_plan (host) checks the table, writes each job's blk0 and returns the
// CTA count and shared memory of the launch; launch_acorr runs the table
// once it is on the device.
cudaError_t acorr_plan(AcorrJob* jobs_h, int n, long long* blocks, size_t* sm);
cudaError_t launch_acorr(const AcorrJob* jobs_d, int n, long long blocks, size_t sm, const double2* twpool,
                         cudaStream_t st);
// The same passes in FP32-pair arithmetic (FP32 datasets): the pointers of
// the jobs then hold FP32 pairs of the same sizes (in_r: the spectrum as
// pairs; in_c / out_c: complex pairs); out_r / out_r32 stay FP64 / FP32.
// twpool: the twiddles as complex FP32 pairs.
cudaError_t launch_acorr_df(const AcorrJob* jobs_d, int n, long long blocks, size_t sm, const void* twpool,
                            cudaStream_t st);

// One forward pass of the count spectrum |F(c_zp)|^2 in FP32-pair arithmetic
// (FP32 datasets), for one dataset: lines O I, element (o, x, i) at
// (o X + x) I + i for x < X (the grid's M_k values along the axis, zero-
// extended to P), its forward DFT of length P, the first Y frequencies kept.
// The first pass reads the FP32 counts (in_f, rows: I = 1) and keeps the
// half spectrum; the others read complex pairs (in_c).  A pass before the
// last writes (o, y, i) at (o Y + y) I + i (out_c); the last (axis 0, O = 1)
// writes |X_y|^2 as an FP32 pair to out_s at q P + y, q the inner index
// (w_1 .. w_{d-1}, extents ext[1..d-1], w_{d-1} fastest) reordered with
// w_{d-1} slowest: the layout the autocorrelation passes read.
struct SpecJob {
    const float* in_f;
    const void* in_c;
    void* out_c;
    void* out_s;
    long long O, I;
    int X, Y, nl, d;
    int ext[MAXD];
    AxisPlan ap;
    long long blk0;
};
cudaError_t spec_plan(SpecJob* jobs_h, int n, long long* blocks, size_t* sm);
cudaError_t launch_spec_df(const SpecJob* jobs_d, int n, long long blocks, size_t sm, const void* twpool,
                           cudaStream_t st);

// ---- kernel density estimate on the grid and mixture cross term (kde.cu)
struct KdeDesc {
    int d;
    long long M[MAXD];
    int L[MAXD];                 // stencil half-widths
    long long ncells, nstencil;  // prod M, prod (2 L_k + 1)
    double lo[MAXD], delta[MAXD];
    double inv_n;
};
struct MixComp {                 // w (2 pi)^{-d/2} |S|^{-1/2} exp(-(x - mu)^T S^-1 (x - mu) / 2)
    double mu[MAXD];
    double lam[MAXD * MAXD];     // S^-1, row stride MAXD
    double nrm;                  // (2 pi)^{-d/2} |S|^{-1/2}
    double w;
};
// out[g] = n^-1 sum_l c[g - l] ktab[l] for every grid node (ktab: the stencil,
// last axis fastest); counts FP32
cudaError_t launch_kde_grid(const float* counts, const KdeDesc& g, const float* ktab, double* out, int nsm,
                            cudaStream_t st);
// partial[b] (b < nblocks) = block b's share of sum_g c_g sum_m (comps[m] at x_g)
cudaError_t launch_mix_dot(const float* counts, const KdeDesc& g, const MixComp* comps, int ncomp, double* partial,
                           int nblocks, cudaStream_t st);

// Binning (binning.cu).  Grid node k along axis a is lo[a] + k delta[a],
// k < M[a].  Counts accumulate into `counts` (zeroed by the caller);
// `outside` counts the points with a coordinate outside [lo, hi] (or NaN),
// which are never binned.
struct GridDesc {
    int d;
    double lo[MAXD];
    double hi[MAXD];
    double delta[MAXD];
    long long M[MAXD];
};

// acc = double (FP64 atomics) or unsigned long long (fixed point: each
// weight is added as round(w * qscale))
template <typename acc>
cudaError_t launch_bin_linear(const double* X, long long n, const GridDesc& g, acc* counts, long long ncells,
                              unsigned long long* outside, double qscale, int nsm, cudaStream_t st);
// dst[i] = (float)(src[i] * unit)
cudaError_t launch_fix_to_f32(const unsigned long long* src, float* dst, long long n, double unit, cudaStream_t st);
cudaError_t launch_bin_simple(const double* X, long long n, const GridDesc& g, int* counts, long long ncells,
                              unsigned long long* outside, int nsm, cudaStream_t st);
template <typename real>
cudaError_t launch_int_to_real(const int* src, real* dst, long long n, cudaStream_t st);
cudaError_t launch_f32_to_f64(const float* src, double* dst, long long n, cudaStream_t st);
// Batched binning of many datasets (FP32 linear binning in fixed point):
// one launch per phase over a job table, each CTA within one job.
//   phase 0: bin the points into the job's fixed-point accumulators
//            (fix, zeroed by the caller) and count the outside points;
//   phase 1: convert the accumulators to FP32 counts;
//   phase 2: the job's mblk block partials of the coordinate sums (mean
//            pass) or, phase 3, of the centred products (mean given).
struct BinJob {
    const double* X;
    long long n, ncells;
    GridDesc g;
    unsigned long long* fix;
    float* counts;
    unsigned long long* outside;
    double* part;          // phase 2: mblk x (d + d^2) sums of x - shift and (x - shift)(x - shift)^T
    double shift[MAXD];    // phase 2: the grid's centre
    int mblk;
    long long blk0;        // set by the launcher
};
cudaError_t launch_bin_many(BinJob* jobs_h, BinJob* jobs_d, int n, int phase, double qscale, cudaStream_t st);
// one-time kernel attributes of the binning launches (before any graph capture)
cudaError_t prepare_binning();

// blocks of the moment launches (at most two per SM)
int moments_blocks(long long n, int nsm);
// one pass: per block b, out[b (d + d^2) + k] = sum of x_k - s_k and
// out[b (d + d^2) + d + a d + c] = sum of (x_a - s_a)(x_c - s_c)
struct Shift {
    double s[MAXD];
};
cudaError_t launch_moments_shifted(const double* X, long long n, int d, const Shift& sh, double* out, int nsm,
                                   cudaStream_t st);

}  // namespace kdefft
