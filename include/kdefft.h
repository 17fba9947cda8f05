/*
 * kdefft.h -- C ABI of the GB300 (sm_103a) library for FFT-based bandwidth
 * selection in multivariate kernel density estimation with unconstrained
 * (full, symmetric positive definite) d x d bandwidth matrices H.
 *
 * Method: Gramacki & Gramacki, "FFT-Based Fast Bandwidth Selector for
 * Multivariate Kernel Density Estimation" (arXiv 1511.07482).  Sec. 4 gives
 * the four steps for the LSCV objective: (1) bin the sample onto a grid,
 * (2) write the binned double sum (Eq. 14) as a convolution of the counts
 * with a kernel-lag array (Eqs. 17-18, truncated to |j_k| <= L_k by Eq. 25-26),
 * (3) evaluate the convolution with a zero-padded d-dimensional FFT
 * (Eqs. 19-23), (4) multiply by the counts and sum (Eq. 24).  Sec. 5 extends
 * the same steps to the functionals psi_r (Eq. 13) and to the scalar
 * eta_{r,s} V-statistics (Eqs. 29-32) used by the SCV and plug-in selectors.
 *
 * Conventions shared by every entry point
 *   - Return value: KDEFFT_OK (0) or one of the KDEFFT_ERR_* codes below;
 *     kdefft_strerror() names a code, kdefft_last_error() gives a one-line
 *     description of the most recent failure on the calling thread.
 *   - Pointers: the caller owns every pointer argument.  Array arguments that
 *     are marked "host or device" may point to host memory or to device
 *     memory of the context's GPU (detected with cudaPointerGetAttributes);
 *     all other arrays are host memory.  Calls are ordered on the stream given
 *     to kdefft_create and return after host outputs have been written;
 *     device outputs are complete when that stream reaches the call's end.
 *   - Layouts: the sample X is n x d FP64 row-major; a bandwidth H (and the
 *     pilot G) is d x d FP64 row-major and must be symmetric to 1e-12
 *     relative (it is symmetrised as (H + H^T)/2) and positive definite (FP64
 *     Cholesky, checked before any launch: KDEFFT_ERR_NOT_SPD).  Batches of
 *     bandwidths are nH consecutive d x d matrices.  Grid counts are laid out
 *     row-major over (M_0, ..., M_{d-1}), last axis fastest.
 *   - Gradients: d x d symmetric FP64 matrices g per bandwidth with
 *     g_aa = dF/dH_aa and, for a != b, g_ab = g_ba = derivative of F along
 *     E_ab + E_ba (the single free off-diagonal parameter moving both entries).
 *   - Limits: 1 <= d <= 4, 2 <= M_k, padded sizes P_k <= 4096 and of the form
 *     2^a 3^b 5^c, derivative order r even and r <= 8 (r <= 6 when d = 4).
 *   - Threads: a context serves one host thread at a time (contexts on
 *     different threads are independent).  Inside a call with thousands of
 *     bandwidths the library may build its requests on up to four host
 *     threads of its own, joined before the call returns; results do not
 *     depend on it.
 */
#ifndef KDEFFT_H
#define KDEFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define KDEFFT_OK               0
#define KDEFFT_ERR_ARG          1  /* bad argument: sizes, d, r, null pointer  */
#define KDEFFT_ERR_NOT_SPD      2  /* H, G or a derived covariance not SPD     */
#define KDEFFT_ERR_OUTSIDE_GRID 3  /* sample point outside [lo, hi] (policy ERROR) */
#define KDEFFT_ERR_CUDA         4  /* a CUDA runtime call failed               */
#define KDEFFT_ERR_ALLOC        5  /* device or host allocation failed         */
#define KDEFFT_ERR_TIMEOUT      6  /* a bounded device-side wait gave up       */
#define KDEFFT_ERR_UNSUPPORTED  7  /* size outside the limits above            */

/* ---- options ------------------------------------------------------------ */
/* Effective-support basis for L_k (Eq. 26): which matrix's largest
 * eigenvalue sets L_k.  AUTO: the bandwidth argument itself for LSCV and
 * psi_r (the paper's rule, lambda_max(H)); the widest covariance in the kernel
 * for SCV (2H + 2G) and for the plug-in functionals (G).  FULL: L_k = M_k - 1
 * (no truncation, Eq. 17). */
enum { KDEFFT_L_AUTO = 0, KDEFFT_L_PAPER = 1, KDEFFT_L_WIDEST = 2, KDEFFT_L_FULL = 3 };
/* Padded FFT length P_k.  MINIMAL: smallest 2^a 3^b 5^c >= M_k + L_k (the
 * least length for which the circular convolution has no wrapped term at the
 * needed outputs).  PAPER: Eq. 27, 2^ceil(log2(M_k + 2 L_k - 1)).
 * PAPER_FULL: Eq. 21, 2^ceil(log2(3 M_k - 1)).  FIXED: opts.P_fixed[k]
 * (must be >= M_k + L_k). */
enum { KDEFFT_P_MINIMAL = 0, KDEFFT_P_PAPER = 1, KDEFFT_P_PAPER_FULL = 2, KDEFFT_P_FIXED = 3 };
enum { KDEFFT_FP32 = 0, KDEFFT_FP64 = 1 };
/* LINEAR: multilinear weights to the 2^d surrounding nodes (Sec. 4 first
 * step).  SIMPLE: weight 1 to the nearest node, ties at half a bin upwards;
 * counts are exact integers. */
enum { KDEFFT_BIN_LINEAR = 0, KDEFFT_BIN_SIMPLE = 1 };
enum { KDEFFT_OUTSIDE_ERROR = 0, KDEFFT_OUTSIDE_DROP = 1 };
enum { KDEFFT_LSCV = 0, KDEFFT_SCV = 1, KDEFFT_PI = 2 };
enum { KDEFFT_DT_F32 = 0, KDEFFT_DT_F64 = 1, KDEFFT_DT_I32 = 2 };

typedef struct {
    double tau;          /* Eq. 26 support multiplier; the paper suggests 3.7 */
    int    L_basis;      /* KDEFFT_L_*                                          */
    int    P_rule;       /* KDEFFT_P_*                                          */
    int    P_fixed[4];   /* used with KDEFFT_P_FIXED                            */
    int    exact_loo;    /* LSCV: 0 = Eq. 10 (n ~ n-1), 1 = Eq. 8 (leave-one- */
                         /* out; needs n >= 2, else KDEFFT_ERR_ARG)           */
    int    precision;    /* KDEFFT_FP32 or KDEFFT_FP64 arithmetic on the GPU    */
    int    binning;      /* KDEFFT_BIN_*                                        */
    int    outside_policy; /* KDEFFT_OUTSIDE_*                                  */
} kdefft_opts;

typedef struct kdefft_ctx_s* kdefft_ctx;
typedef struct kdefft_ds_s*  kdefft_ds;

/* Fill *opts with the defaults: tau 3.7, L AUTO, P MINIMAL, exact_loo 0,
 * FP32, LINEAR binning, outside points are an error. */
int kdefft_opts_default(kdefft_opts* opts);

/* Create a context on CUDA device `device`, ordering all work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Inside a call some
 * launches may run on a second stream of the context's own, forked from
 * `stream` after the work before them and joined back into it before the
 * call's later work: the ordering on `stream` is unchanged.  The context
 * owns its device buffers (twiddle tables, scratch, work lists) until
 * kdefft_destroy.
 * Fails with KDEFFT_ERR_CUDA when no usable GPU is present: there is no CPU
 * fallback. */
int kdefft_create(kdefft_ctx* ctx, int device, void* stream);
/* Destroy a context and every dataset still open on it.  A handle that is
 * not live (destroyed already, or never created) is KDEFFT_ERR_ARG; NULL is
 * a no-op.  The same holds for kdefft_ds_destroy. */
int kdefft_destroy(kdefft_ctx ctx);

/* Step 1 of Sec. 4: bin the sample X (n x d FP64 row-major; host or device)
 * onto the grid g_k1 = lo[k] .. g_kM_k = hi[k] with M[k] nodes per axis
 * (bin width Eq. 16).  Creates a dataset that owns the device counts and the
 * cached count spectra |F(c_zp)|^2 (one per padded size) until
 * kdefft_ds_destroy.  opts may be NULL (defaults); the dataset keeps a copy.
 * Points outside the grid: KDEFFT_ERR_OUTSIDE_GRID under policy ERROR (no
 * dataset is created), skipped under policy DROP (n keeps its value as the
 * sample size; kdefft_ds_info reports the dropped count). */
int kdefft_bin(kdefft_ctx ctx, const double* X, int64_t n, int d,
               const double* lo, const double* hi, const int64_t* M,
               const kdefft_opts* opts, kdefft_ds* out);

/* kdefft_bin for nds datasets of the same d at once (Sec. 4 step 1 for
 * each): X[i] is dataset i's n[i] x d sample (host or device), lo/hi its
 * grid range (nds x d), M its grid (nds x d).  FP32 linear binning runs as
 * three launches over all datasets (binning, conversion, the one-pass
 * covariance) with one synchronisation in total, and the datasets' counts
 * share one allocation (freed with the last of them); other precisions and
 * rules bin one dataset at a time.  out: nds handles.  On error no dataset
 * is created. */
int kdefft_bin_many(kdefft_ctx ctx, int nds, const double* const* X, const int64_t* n, int d,
                    const double* lo, const double* hi, const int64_t* M, const kdefft_opts* opts,
                    kdefft_ds* out);
int kdefft_ds_destroy(kdefft_ds ds);

/* Replace the dataset's per-call options (tau, L_basis, P_rule, P_fixed,
 * exact_loo).  Precision, binning and outside policy are fixed at bin time
 * and are ignored here. */
int kdefft_ds_set_opts(kdefft_ds ds, const kdefft_opts* opts);

/* n (sample size), d, and the number of dropped points. */
int kdefft_ds_info(kdefft_ds ds, int64_t* n, int* d, int64_t* dropped);

/* Copy the grid counts (prod M_k values) to dst (host or device) as dtype
 * KDEFFT_DT_F32, _F64 or _I32 (I32 only for SIMPLE binning, exact). */
int kdefft_counts(kdefft_ds ds, void* dst, int dtype);

/* The truncation L_k (Eq. 26) and padded sizes P_k that the functional
 * `method` (KDEFFT_LSCV, _SCV, _PI) or, when method < 0, psi_r would use for
 * bandwidth H (and pilot G where the method takes one); d ints each. */
int kdefft_plan(kdefft_ds ds, int method, const double* H, const double* G,
                int* L_out, int* P_out);

/* psi_r(H) of Eq. 13 with the Gaussian kernel, binned (Eq. 25) and
 * evaluated by Secs. 4-5's FFT steps, for nH bandwidths: out holds nH
 * vectors of d^r FP64 values in Kronecker order (Sec. 5: position
 * (i_1..i_r), i_1 slowest, holds n^-2 sum_ij d^alpha phi_H(X_i - X_j) with
 * alpha_k = #{m : i_m = k}).  r even, 0 <= r <= 8.  out: host or device. */
int kdefft_psi(kdefft_ds ds, const double* H, int nH, int r, double* out);

/* Adjoint of psi_r (Eq. 13) for reverse-mode differentiation: for each of
 * the nH bandwidths H_k, out_k = sum_i w_{k,i} d psi_{r,i}(H_k) / d H, a d x d
 * matrix whose entry (a, b) is the derivative in H_ab with the d^2 entries of
 * H taken as independent (evaluated at the symmetric H; each off-diagonal
 * entry gets half the tied derivative of the other calls).  By the Gaussian's
 * heat equation d phi_H / dH = 1/2 grad grad^T phi_H (Sec. 5's derivative
 * functionals), d psi_alpha / d H_ab = 1/2 psi_{alpha + e_a + e_b}, so this
 * evaluates psi_{r+2} at each H (binned, the same FFT steps as kdefft_psi)
 * and contracts it with w.  w: nH x d^r (Kronecker order, as kdefft_psi's
 * output), host or device; out: nH x d x d FP64, host or device.  Errors:
 * KDEFFT_ERR_UNSUPPORTED when r + 2 exceeds the order limit for d. */
int kdefft_psi_grad(kdefft_ds ds, const double* H, int nH, int r, const double* w, double* out);

/* LSCV(H) for nH bandwidths: Eq. 10 (psi of Eq. 12 with T_H of Eq. 11, plus
 * 2 n^-1 K_H(0)) or, with opts.exact_loo, Eq. 8.  val: nH FP64; grad: NULL
 * or nH d x d gradients (heat-equation kernels through the same FFT, L held
 * at the value's L).  val/grad: host or device. */
int kdefft_lscv(kdefft_ds ds, const double* H, int nH, double* val, double* grad);

/* SCV(H) with pilot G (d x d), Gaussian kernels, V-statistic form:
 * n^-1 (4 pi)^{-d/2} |H|^{-1/2} + n^-2 sum_ij [phi_{2H+2G} - 2 phi_{H+2G}
 * + phi_{2G}](X_i - X_j).  The paper names SCV (Sec. 3) and defers its
 * formula (Sec. 5) to Chacon & Duong; this is that source's Gaussian form.
 * The three Gaussian sums are reduced separately and combined in FP64 (the
 * full kernel integrates to zero); the phi_2G sum depends on G, L and P
 * only and is cached on the dataset.  val/grad as kdefft_lscv. */
int kdefft_scv(kdefft_ds ds, const double* H, int nH, const double* G,
               double* val, double* grad);

/* Plug-in objective PI(H) = n^-1 (4 pi)^{-d/2} |H|^{-1/2} + 1/4 (vec^T H)^{(x)2}
 * psi_4(G) with pilot G: the fourth-order functional psi_4(G) is computed
 * once per call (binned, FFT) and contracted per H; equivalently the
 * eta_{0,2}(.; H, G) V-statistic of Eqs. 29-30.  val/grad as kdefft_lscv. */
int kdefft_pi(kdefft_ds ds, const double* H, int nH, const double* G,
              double* val, double* grad);

/* Per-H plug-in functional V = n^-2 sum_ij eta_{0,2}(X_i - X_j; H, G)
 * (Eq. 29 with Eq. 30, r = 0, s = 2): one scalar kernel grid per H through
 * the FFT.  val: nH FP64, host or device. */
int kdefft_eta02(kdefft_ds ds, const double* H, int nH, const double* G, double* val);

/* V-statistic Q_r(Sigma) = n^-2 sum_ij eta(X_i - X_j; Sigma) (Eq. 32) with
 * eta = Laplacian^{r/2} phi_Sigma = (vec^T I)^{(x) r/2} D^{(x) r} phi_Sigma
 * (Eq. 31's eta_{r/2}): r is the total derivative order, even, at most the
 * order limit for d (8 for d <= 3, 6 for d = 4).  One value per Sigma (nS
 * row-major d x d SPD matrices); support from lambda_max(Sigma) (Eq. 26).
 * out: nS FP64, host or device. */
int kdefft_qr(kdefft_ds ds, const double* Sigma, int nS, int r, double* out);

/* V-statistic of Eq. 29, n^-2 sum_ij eta_{r,s}(X_i - X_j; A, B, Sigma), with
 * eta_{r,s} = {(vec^T A)^{(x)r} (x) (vec^T B)^{(x)s}} D^{(x)2r+2s} phi_Sigma
 * (Eq. 30), the building block of the plug-in and SCV selectors for density
 * derivative estimation.  A, B: symmetric d x d (NULL: the identity);
 * Sigma: nS SPD d x d; 2(r + s) at most the order limit for d and at most
 * 40 distinct partials.  eta_{0,2} with B = H, Sigma = G is kdefft_eta02;
 * A = I, s = 0 is the eta of kdefft_qr with order 2r.  out: nS FP64, host or
 * device. */
int kdefft_eta_rs(kdefft_ds ds, const double* A, const double* B, const double* Sigma, int nS, int r, int s,
                  double* out);

/* The binned kernel density estimate (Eq. 1 with the sample replaced by its
 * bin counts) at every grid node: f_hat(g) = n^-1 sum_{|l_k| <= L_k}
 * c_{g-l} K_H(delta (.) l), the convolution that the FFT steps of Sec. 4
 * evaluate, truncated at the support L of Eq. 26 (from lambda_max(H)).
 * out: prod M_k FP64, row-major over the grid (last axis fastest), host or
 * device.  FP32 linear-binned datasets (else KDEFFT_ERR_UNSUPPORTED). */
int kdefft_kde_grid(kdefft_ds ds, const double* H, double* out);

/* Integrated squared error (Eq. 37) of the binned estimate against a normal
 * mixture f = sum_m w_m phi_{S_m}(. - mu_m), in closed form:
 *   int f_hat^2 = n^-2 sum_ij phi_2H(g_i - g_j) c_i c_j (the binned double
 *                 sum, as every functional here),
 *   int f_hat f = n^-1 sum_g c_g sum_m w_m phi_{H + S_m}(x_g - mu_m),
 *   int f^2     = sum_lm w_l w_m phi_{S_l + S_m}(mu_l - mu_m),
 * ISE = the first - 2 the second + the third.  K in 1..64 components; w: K;
 * mu: K x d; S: K x d x d SPD.  out: nH FP64, host or device.  FP32
 * linear-binned datasets. */
int kdefft_ise_mixture(kdefft_ds ds, const double* H, int nH, int K, const double* w, const double* mu,
                       const double* S, double* out);

/* LSCV_r(H) for estimating the r-th density derivative (Eq. 36; with the
 * dataset's exact_loo option, Eq. 35), with eta_{r,0}(.; H) = Laplacian^r
 * phi_H, kernels of order 2r (2r at most the order limit for d).  The
 * n ~ n-1 form adds 2 n^-1 eta_r(0; H) (reading of Eq. 36's last term,
 * which is 2 n^-1 K_H(0) at r = 0).  Values only.  val: nH FP64, host or
 * device. */
int kdefft_lscv_r(kdefft_ds ds, const double* H, int nH, int r, double* val);

/* Minimise `method` (KDEFFT_LSCV or _SCV or _PI) over H in F, the SPD
 * matrices (Eq. 9), with a quasi-Newton method on the Cholesky factor of H
 * (log diagonal) using the exact gradients.  H0: start (NULL: the normal-scale
 * rule (4/(d+2))^{2/(d+4)} n^{-2/(d+4)} S_hat).  G: pilot for SCV/PI (NULL:
 * the normal-scale matrix).  n_starts >= 1 independent starts (start 0 is H0,
 * the others are deterministic dilations/rotations of it) run in lock-step,
 * one batched evaluation per iteration; the best end point is returned.
 * H_out: d x d; f_out: objective at H_out; n_evals: total objective+gradient
 * evaluations (may be NULL). All host.  Search domain: H numerically SPD
 * with sqrt(H_kk) >= delta_k / 2 (bandwidths finer than half a bin are not
 * resolved by the binned objective, which is unbounded below as H -> 0 when
 * bins hold several points); trial points outside it are rejected by the line
 * search.  Steps change the Cholesky diagonal by at most a factor e. */
int kdefft_select_H(kdefft_ds ds, int method, const double* H0, const double* G,
                    int n_starts, int max_iter, double* H_out, double* f_out,
                    int64_t* n_evals);

/* Several criteria minimised on one dataset: methods[m] (KDEFFT_LSCV, _SCV
 * or _PI) for m < nmethods, each with the arguments and the result of
 * kdefft_select_H (the same starts from H0, the same G).  H_out: nmethods x
 * d x d; f_out and n_evals: nmethods each (may be NULL).  Where the
 * device-resident d = 2 search covers two of the criteria they run in one
 * launch, one CTA per start of either, against one autocorrelation box
 * sized for both; the others run one after another.  Every result is the
 * one kdefft_select_H gives for that criterion on a dataset whose
 * autocorrelation box is already this large. */
int kdefft_select_H_multi(kdefft_ds ds, int nmethods, const int* methods, const double* H0, const double* G,
                          int n_starts, int max_iter, double* H_out, double* f_out, int64_t* n_evals);

/* Bandwidth classes (Sec. 3): F, full SPD matrices (the paper's subject);
 * D, diagonal matrices; S, scalar multiples h^2 I of the identity. */
enum { KDEFFT_H_FULL = 0, KDEFFT_H_DIAG = 1, KDEFFT_H_SCALAR = 2 };

/* kdefft_select_H (optimizer 0) or kdefft_select_H_nm (optimizer 1) with H
 * restricted to a class: D searches the log square roots of the diagonal,
 * S the log of h; starts are the class projections of the usual starts
 * (the diagonal of each start for D, h^2 = the geometric mean of its
 * diagonal for S).  The device-resident d = 2 search covers F only; D and S
 * run the host-driven search.  Same arguments, domain and errors otherwise. */
int kdefft_select_H_class(kdefft_ds ds, int method, int hclass, int optimizer, const double* H0, const double* G,
                          int n_starts, int max_iter, double* H_out, double* f_out, int64_t* n_evals);

/* The same minimisation with the derivative-free Nelder-Mead method the
 * paper's experiments use (Sec. 6: reflection 1.0, contraction 0.5,
 * expansion 2.0), for parity with its selections.  Simplex in the same
 * Cholesky parameters theta (log diagonal), initial vertices theta_0 and
 * theta_0 + 0.1 e_i; shrink towards the best vertex by the contraction
 * factor; stop when f_worst - f_best <= 2^-26 (|f_best| + 2^-26) or after
 * max_iter objective evaluations per start (max_iter < 1: 500).  Only
 * objective values are evaluated.  Same arguments, domain, starts and
 * errors as kdefft_select_H. */
int kdefft_select_H_nm(kdefft_ds ds, int method, const double* H0, const double* G,
                       int n_starts, int max_iter, double* H_out, double* f_out,
                       int64_t* n_evals);

/* LSCV(H) and its gradient for many datasets at once: dataset i gets
 * nH_per_ds[i] consecutive bandwidths from H; every (dataset, H) unit runs
 * in one batched launch sequence.  val: total nH FP64; grad: NULL or total
 * nH d x d.  All datasets must belong to ctx and share d and precision.
 * H, val, grad: host. */
int kdefft_batch_lscv(kdefft_ctx ctx, int nds, const kdefft_ds* ds,
                      const int* nH_per_ds, const double* H,
                      double* val, double* grad);

/* Engine selection.  AUTO (default): a grid whose padding has no aliasing
 * (P_k >= M_k + L_k on every axis, which every P rule but a small FIXED size
 * gives) is evaluated in the lag domain: n^-2 sum_j w_j k_j a_j over the half
 * support box, with the count autocorrelation a = F^-1(|C|^2) computed once
 * per dataset in FP64 -- Eq. 25 summed over the lag first, the same value as
 * the FFT route of Eqs. 19-24.  Other grids take the FFT route: for d = 2 one
 * thread-block-cluster kernel per batch does all passes in shared and
 * distributed shared memory whenever the work fits, else the multi-pass
 * path.  kdefft_select_H on a d = 2 FP32 dataset (LSCV of Eq. 10 or SCV,
 * minimal padding) runs the whole multi-start search in one device-resident
 * launch (one cluster per start).  HOST_SELECT: as AUTO but the search is
 * driven from the host, one batched launch per round.  FFT: as AUTO without
 * the lag domain.  MULTIPASS: only the pass-per-axis FFT kernels with a
 * global scratch between passes, host-driven search.  All compute the same
 * sums. */
enum {
    KDEFFT_ENGINE_AUTO = 0,
    KDEFFT_ENGINE_MULTIPASS = 1,
    KDEFFT_ENGINE_HOST_SELECT = 2,
    KDEFFT_ENGINE_FFT = 3
};
int kdefft_set_engine(kdefft_ctx ctx, int engine);

/* Autotuner (off by default).  When on, the first batch of each shape
 * (dimension, precision, and the number of work items, largest padded size
 * and largest support, each rounded up to a power of two) is run once per
 * candidate configuration -- engine (fused cluster kernel for d = 2 /
 * multi-pass), multi-pass tile capacity (1/2, 1 and 3/2 of the default
 * lines x padded size per CTA batch), largest FFT radix (32 or 16 in FP32,
 * 16 or 8 in FP64) -- each timed on the host clock over the whole batch;
 * the fastest is kept for the shape and its results are the batch's.  Later
 * batches of the shape use it directly.  Results of different candidates
 * agree within the FP32 (FP64) tolerance of the evaluation. */
int kdefft_set_autotune(kdefft_ctx ctx, int on);

/* The count autocorrelation a_j = sum_i c_i c_{i+j} (the lag-domain form of
 * Eq. 25's double sum) on the half box j_0 in [0, A_0], |j_k| <= A_k
 * (k >= 1), A_k <= M_k - 1: out holds prod_{k>=1} (2 A_k + 1) x (A_0 + 1)
 * FP64 values, layout [j_{d-1}]..[j_1][j_0] (j_0 fastest, index j_k + A_k
 * for k >= 1); a_{-j} = a_j gives the other half.  Computed in FP64 from the
 * count spectrum at the smallest 2^a 3^b 5^c padding >= M_k + A_k (cached on
 * the dataset and reused by the lag-domain engine).  out: host.  Errors:
 * KDEFFT_ERR_ARG for A outside [0, M_k - 1], KDEFFT_ERR_UNSUPPORTED when that
 * padding exceeds 4096 on an axis. */
int kdefft_autocorr(kdefft_ds ds, const int* A, double* out);

/* CUDA graphs (on by default).  A batch's launch sequence (staging copy,
 * kernels, result copy) is captured once into a CUDA graph under its
 * launch signature -- every device and pinned-host pointer, size, tile
 * count and launch shape -- and replayed when a later batch has the same
 * signature (the work items themselves are data read at replay time).  At
 * most 64 graphs per context; the cache is emptied when full.  Disabled while
 * profiling is on (kdefft_profile), so that each kernel keeps its own CUDA
 * events. */
int kdefft_set_graphs(kdefft_ctx ctx, int on);

/* Record of the device-resident searches' own evaluations (Eq. 9's
 * minimiser on the d = 2 FP32 path of kdefft_select_H and
 * kdefft_select_H_multi), so that each value and gradient the search compares
 * can be checked against an FP64 evaluation at the same bandwidth.  rec: a
 * device buffer on the context's GPU of rec_len doubles, or NULL to turn
 * recording off (the default; the search kernels then write nothing).  While
 * on, the s-th start of a search launch (criteria in the order given to
 * kdefft_select_H_multi, each criterion's starts in order) writes its e-th
 * evaluation, for e < cap, to rec[(s cap + e) 12 ..] as 12 doubles: s, e,
 * criterion (0 LSCV of Eq. 10, 1 SCV), H_00, H_01, H_11 (the FP32 values the
 * search evaluated), L_0, L_1 (Eq. 26, as the search computed them), the
 * objective value, and its gradient dF/dH_00, dF/dH_01 (tied convention),
 * dF/dH_11.  Slots of evaluations that did not happen are left untouched.
 * The caller keeps the buffer alive while recording is on; a search with
 * more than rec_len / (12 cap) starts fails with KDEFFT_ERR_ARG before its
 * launch.  Errors: KDEFFT_ERR_ARG (cap < 1, rec_len < 12 cap, rec not device
 * memory of the context's GPU). */
int kdefft_set_search_record(kdefft_ctx ctx, double* rec, int64_t rec_len, int cap);

/* Counters of the two above since the context was created: shapes tuned,
 * graphs captured, graph replays.  Any pointer may be NULL. */
int kdefft_runtime_stats(kdefft_ctx ctx, int64_t* shapes_tuned,
                         int64_t* graphs_captured, int64_t* graph_replays);

/* Device memory of datasets.  Blocks a destroyed dataset (or a growing
 * buffer of one) held go back to a per-context cache and serve later
 * datasets of the context, in the order of its stream, so that binning a
 * dataset per step allocates nothing once the cache holds blocks of the
 * sizes needed.  At most 16 GiB stay cached (the largest free blocks beyond
 * that are released); an allocation that fails releases the cache and
 * retries once.  kdefft_memory_stats: bytes held in free blocks, blocks
 * served from the cache, blocks allocated from CUDA (any pointer may be
 * NULL).  kdefft_trim releases every free block (synchronising the device,
 * as cudaFree does).  The context releases them when destroyed. */
int kdefft_memory_stats(kdefft_ctx ctx, int64_t* cached_bytes, int64_t* hits, int64_t* misses);
int kdefft_trim(kdefft_ctx ctx);

/* LSCV value and gradient for one bandwidth without allocating any memory.
 * The paper has no counterpart: this is for callers that cannot allocate at
 * the point of the call -- code that runs under a device-memory budget fixed
 * in advance, code called back from inside another framework's allocator, or
 * latency-critical loops where a cudaMalloc (which synchronises the device and
 * can fail) is not acceptable.  It calls no cudaMalloc, cudaFree or other
 * allocating routine; its work buffers live in one scratch array of
 * KDEFFT_NOALLOC_SCRATCH_BYTES (32 MiB) inside the library image, which every
 * GPU that loads the library holds until the process exits.
 *   d: 1..3; M: d grid sizes; delta: d bin widths (Eq. 16); n: sample size;
 *   counts: device pointer to prod M_k FP32 grid counts, row-major (e.g. from
 *   kdefft_counts); H: d x d host array; tau: Eq. 26 multiplier (L_k from
 *   lambda_max(H)); P_k: the minimal no-alias padding; stream: cudaStream_t;
 *   out: device pointer to 1 + d*d FP64 values, LSCV(H) of Eq. 10 followed by
 *   the d x d gradient (convention above).  counts and out must be device
 *   memory of the calling thread's current device.
 * Runs on the current device and is ordered on `stream`; the host does not
 * wait for the kernels, but its small tables go up by copies from pageable
 * host memory, so a call may wait for earlier work on its stream.  The first
 * call on a device takes the scratch array's device address
 * (cudaGetSymbolAddress), uploads small constant tables and sets the
 * kernels' shared-memory limits.  While `stream` is being captured the call
 * does nothing and returns KDEFFT_ERR_UNSUPPORTED: those uploads read host
 * staging that the next call overwrites.  All calls share the one scratch
 * array, which keeps the previous call's contents (everything that must
 * start at zero is written before it is read), so calls that overlap on the
 * GPU -- on different streams, unordered -- race; order them on one stream.
 * Errors: KDEFFT_ERR_ARG (bad sizes, out/counts not device memory of the
 * current device, H not symmetric), KDEFFT_ERR_NOT_SPD,
 * KDEFFT_ERR_UNSUPPORTED (the problem needs more than the scratch array
 * holds, P_k > 4096, or the stream is being captured), KDEFFT_ERR_CUDA. */
#define KDEFFT_NOALLOC_SCRATCH_BYTES (32u << 20)
int kdefft_lscv_noalloc(int d, const int64_t* M, const double* delta, int64_t n,
                        const float* counts, const double* H, double tau,
                        void* stream, double* out);

/* The radix schedule of the library's 1-D transforms of length P (Eqs.
 * 19-22 on each axis): the fewest Stockham stages whose radices (at most
 * max_radix; 2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32)
 * multiply to P, in the order the passes apply them.  radices: room for 16
 * ints; *nstages receives their count.  Needs no GPU; shared by every
 * context (the schedule cache is thread-safe).  Errors: KDEFFT_ERR_UNSUPPORTED
 * for P outside [2, 4096] or not of the form 2^a 3^b 5^c. */
int kdefft_radix_plan(int P, int max_radix, int* radices, int* nstages);

/* Instrumentation (no paper counterpart).  kdefft_profile(ctx, mode):
 * mode 1 resets the counters and turns per-kernel timing on, 2 turns it on
 * without a reset, 0 resets and turns it off.  With timing on, every kernel
 * launch of the context is bracketed by CUDA events on the context's stream
 * and its algorithmic bytes (the bytes the pass must move: inputs read once,
 * outputs written once) and FFT flops (5 P log2 P per transformed line) are
 * accumulated per kernel name.  Kernel launches and host<->device bytes are
 * always counted.  kdefft_profile_read copies up to `cap` records. */
typedef struct {
    char    name[24];
    int64_t launches;
    double  ms;        /* summed CUDA-event duration of the launches */
    double  bytes;     /* summed algorithmic bytes                   */
    double  flops;     /* summed algorithmic flops                   */
} kdefft_kstat;

int kdefft_profile(kdefft_ctx ctx, int mode);
int kdefft_profile_read(kdefft_ctx ctx, kdefft_kstat* out, int cap, int* count,
                        int64_t* launches, int64_t* h2d_bytes, int64_t* d2h_bytes);

const char* kdefft_strerror(int code);
const char* kdefft_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KDEFFT_H */
