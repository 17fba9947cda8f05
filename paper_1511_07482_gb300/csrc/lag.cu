// Lag-domain evaluation of the binned functionals (Eq. 25 with the sum over
// the lag done first) and the count autocorrelation it needs.
//
//   acorr_axis  one pass of the pruned inverse DFT a = F^-1(|C|^2) (FP64):
//               the count spectrum of Eq. 22 at a padded size P >= M + A has
//               no aliasing at lags |j_k| <= A_k, so a_j = sum_i c_i c_{i+j}
//               exactly (up to rounding) on that box.
//   lag         per work item (two kernels of the same covariances and
//               support, as in the FFT path), sum over the half lag box of
//               w_j k_j a_j, w_j in {0, 1, 2}; kernels from the
//               compile-time Hermite recurrence; compensated FP32 (or FP64)
//               sums, one FP64 partial per tile.
//   lag_reduce  fixed-order sum of an item's tile partials, times n^-2.
#include <algorithm>

#include "devutil.cuh"
#include "engine.cuh"

namespace kdefft {

// ------------------------------------------------------------ autocorrelation passes
// twiddles exp(-2 pi i t / P) of one size in shared memory when they fit
constexpr int kTwSmem = 2048;

// the job owning block b (jobs in increasing blk0)
__device__ __forceinline__ int acorr_job_of(const AcorrJob* __restrict__ jobs, int n, long long b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].blk0 <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Innermost axis of the real spectrum (layout [o][w], one row of W values
// per o): one CTA per (job, row), the row and the twiddles staged in shared
// memory, one warp per output lag, the lanes splitting the sum.
__global__ void __launch_bounds__(256) k_acorr_row(const AcorrJob* __restrict__ jobs, int njobs,
                                                   const double2* __restrict__ twpool) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const AcorrJob& jb = jobs[acorr_job_of(jobs, njobs, blockIdx.x)];
    const long long o = (long long)blockIdx.x - jb.blk0;
    const int P = jb.P, W = jb.W, J = jb.J;
    const bool tws = P <= kTwSmem;
    double2* stw = reinterpret_cast<double2*>(sm_raw);
    double* row = reinterpret_cast<double*>(stw + (tws ? P : 0));
    const double2* tw = twpool + jb.tw_off;
    if (tws)
        for (int t = threadIdx.x; t < P; t += blockDim.x) stw[t] = tw[t];
    for (int w = threadIdx.x; w < W; w += blockDim.x) row[w] = jb.in_r[o * W + w];
    __syncthreads();
    const double2* T = tws ? stw : tw;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int jj = warp; jj < J; jj += nw) {
        int step = (jb.jlo + jj) % P;
        if (step < 0) step += P;
        // position (w step) mod P for w = lane, lane + 32, ...
        int pos = (int)(((long long)lane * step) % P);
        const int adv = (int)((32LL * step) % P);
        double sr = 0.0, si = 0.0;
        for (int w = lane; w < W; w += 32) {
            const double2 t = T[pos];
            const double h = (jb.half && w != 0 && 2 * w != P) ? 2.0 : 1.0;
            const double x = h * row[w];
            sr = fma(x, t.x, sr);
            si = fma(-x, t.y, si);
            pos += adv;
            if (pos >= P) pos -= P;
        }
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) {
            sr += __shfl_down_sync(0xffffffffu, sr, sh);
            si += __shfl_down_sync(0xffffffffu, si, sh);
        }
        if (lane == 0) {
            const long long idx = o * J + jj;
            if (jb.out_r) {
                jb.out_r[idx] = sr * jb.scale;
                if (jb.out_r32) jb.out_r32[idx] = (float)(sr * jb.scale);
            } else {
                jb.out_c[idx] = make_double2(sr, si);
            }
        }
    }
}

// Outer axis of complex data [o][w][i] -> [o][jj][i]: one thread per output,
// i fastest (coalesced reads, one twiddle per warp and step), each CTA within
// one job, twiddles in shared memory.
__global__ void __launch_bounds__(256) k_acorr_axis(const AcorrJob* __restrict__ jobs, int njobs,
                                                    const double2* __restrict__ twpool) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const AcorrJob& jb = jobs[acorr_job_of(jobs, njobs, blockIdx.x)];
    const int P = jb.P, W = jb.W, J = jb.J;
    const long long I = jb.I;
    const bool tws = P <= kTwSmem;
    double2* stw = reinterpret_cast<double2*>(sm_raw);
    const double2* tw = twpool + jb.tw_off;
    if (tws) {
        for (int t = threadIdx.x; t < P; t += blockDim.x) stw[t] = tw[t];
        __syncthreads();
    }
    const double2* T = tws ? stw : tw;
    const long long total = jb.O * (long long)J * I;
    const long long idx = ((long long)blockIdx.x - jb.blk0) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const long long i = idx % I;
    const long long r = idx / I;
    const int jj = (int)(r % J);
    const long long o = r / J;
    int step = (jb.jlo + jj) % P;
    if (step < 0) step += P;
    int pos = 0;
    double sr = 0.0, si = 0.0;
    const long long base = o * (long long)W * I + i;
    for (int w = 0; w < W; ++w) {
        const double2 t = T[pos];   // exp(-2 pi i pos / P); the pass uses its conjugate
        const double2 x = jb.in_c[base + (long long)w * I];
        const double h = (jb.half && w != 0 && 2 * w != P) ? 2.0 : 1.0;
        sr = fma(h * x.x, t.x, fma(h * x.y, t.y, sr));
        si = fma(h * x.y, t.x, fma(-h * x.x, t.y, si));
        pos += step;
        if (pos >= P) pos -= P;
    }
    if (jb.out_r) {
        jb.out_r[idx] = sr * jb.scale;
        if (jb.out_r32) jb.out_r32[idx] = (float)(sr * jb.scale);
    } else {
        jb.out_c[idx] = make_double2(sr, si);
    }
}

cudaError_t launch_acorr_many(AcorrJob* jobs_h, AcorrJob* jobs_d, int n, bool inner, const double2* twpool,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long blocks = 0;
    size_t sm = 0;
    for (int k = 0; k < n; ++k) {
        AcorrJob& jb = jobs_h[k];
        jb.blk0 = blocks;
        const size_t twb = (jb.P <= kTwSmem) ? sizeof(double2) * (size_t)jb.P : 0;
        if (inner) {
            if (jb.I != 1 || !jb.in_r) return cudaErrorInvalidValue;
            blocks += jb.O;
            sm = std::max(sm, twb + sizeof(double) * (size_t)jb.W);
        } else {
            blocks += (jb.O * (long long)jb.J * jb.I + 255) / 256;
            sm = std::max(sm, twb);
        }
    }
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyAsync(jobs_d, jobs_h, sizeof(AcorrJob) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    static size_t set_row = 48 * 1024, set_axis = 48 * 1024;
    size_t& set = inner ? set_row : set_axis;
    if (sm > set) {
        e = cudaFuncSetAttribute(inner ? (const void*)k_acorr_row : (const void*)k_acorr_axis,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        set = sm;
    }
    if (inner)
        k_acorr_row<<<(unsigned)blocks, 256, sm, st>>>(jobs_d, n, twpool);
    else
        k_acorr_axis<<<(unsigned)blocks, 256, sm, st>>>(jobs_d, n, twpool);
    return cudaGetLastError();
}

// ------------------------------------------------------------ lag evaluation
template <typename real, int D, int R>
__global__ void __launch_bounds__(256) k_lag(const LagItem<real>* __restrict__ items,
                                             const LagTile* __restrict__ tiles, int ntiles,
                                             const real* __restrict__ wpool, double* __restrict__ partial) {
    constexpr HTab<D, R> ht{};
    constexpr int N = HTab<D, R>::N;
    __shared__ real Ws[2][MAXSIG][N];
    __shared__ LagItem<real> it;
    for (int tix = blockIdx.x; tix < ntiles; tix += gridDim.x) {
        const LagTile tl = tiles[tix];
        __syncthreads();   // the previous tile's readers of it / Ws are done
        if (threadIdx.x == 0) it = items[tl.item];
        __syncthreads();
        const int nsig = it.nsig;
        for (int t = threadIdx.x; t < 2 * MAXSIG * N; t += blockDim.x) {
            const int h = t / (MAXSIG * N);
            const int s = (t / N) % MAXSIG;
            const int k = t % N;
            (&Ws[0][0][0])[t] = (s < nsig) ? wpool[it.w_off + (h * nsig + s) * N + k] : real(0);
        }
        __syncthreads();
        SumAcc<real> acc;
        const int n0 = it.L[0] + 1;
        const long long end = tl.first + tl.n;
        for (long long f = tl.first + threadIdx.x; f < end; f += blockDim.x) {
            int j[D];
            long long g = f;
            j[0] = (int)(g % n0);
            g /= n0;
#pragma unroll
            for (int k = 1; k < D; ++k) {
                const int w = 2 * it.L[k] + 1;
                j[k] = (int)(g % w) - it.L[k];
                g /= w;
            }
            // half-space weight: 2 where the first nonzero coordinate is positive
            int wt = 1, decided = 0;
#pragma unroll
            for (int k = 0; k < D; ++k)
                if (!decided && j[k] != 0) {
                    wt = j[k] > 0 ? 2 : 0;
                    decided = 1;
                }
            if (wt == 0) continue;
            long long ai = 0;
#pragma unroll
            for (int k = D - 1; k >= 1; --k) ai = ai * (2 * it.A[k] + 1) + (j[k] + it.A[k]);
            ai = ai * (it.A[0] + 1) + j[0];
            const real av = it.acorr[ai];
            real x[D];
#pragma unroll
            for (int k = 0; k < D; ++k) x[k] = it.delta[k] * (real)j[k];
            real va = 0, vb = 0;
#pragma unroll
            for (int s = 0; s < MAXSIG; ++s) {
                if (s < nsig) {
                    real z[D];
                    real q = 0;
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        real zz = 0;
#pragma unroll
                        for (int b = 0; b < D; ++b) zz += it.lam[s][a * MAXD + b] * x[b];
                        z[a] = zz;
                        q += x[a] * zz;
                    }
                    const real e = it.nrm[s] * exp(real(-0.5) * q);
                    real He[N];
                    He[0] = real(1);
#pragma unroll
                    for (int t = 1; t < N; ++t) {
                        real v = z[ht.piv[t]] * He[ht.par[t]];
#pragma unroll
                        for (int r = 0; r < D; ++r)
                            if (r < ht.nred[t])
                                v -= real(ht.rc[t][r]) * it.lam[s][ht.piv[t] * MAXD + ht.rj[t][r]] * He[ht.ridx[t][r]];
                        He[t] = v;
                    }
                    real pa = 0, pb = 0;
#pragma unroll
                    for (int t = 0; t < N; ++t) {
                        pa += Ws[0][s][t] * He[t];
                        pb += Ws[1][s][t] * He[t];
                    }
                    va += e * pa;
                    vb += e * pb;
                }
            }
            const real wa = real(wt) * av;
            acc.add(wa * va, wa * vb);
        }
        double out2[2];
        block_reduce_acc(acc, out2);
        if (threadIdx.x == 0) {
            partial[2 * (long long)tix] = out2[0];
            partial[2 * (long long)tix + 1] = out2[1];
        }
    }
}

template <typename real>
__global__ void k_lag_reduce(const LagItem<real>* __restrict__ items, int nitems, const double* __restrict__ partial,
                             double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nitems) return;
    const LagItem<real>& it = items[i];
    double a = 0.0, b = 0.0;
    for (int t = 0; t < it.ntile; ++t) {
        a += partial[2 * (long long)(it.tile0 + t)];
        b += partial[2 * (long long)(it.tile0 + t) + 1];
    }
    out[2 * i] = a * it.scale;
    out[2 * i + 1] = b * it.scale;
}

// instantiated (d, R): FP32 d <= 2 up to R = 8, d = 3 up to 6, d = 4 up to 4;
// FP64 the same except d = 3 up to 4 (register budget of the Hermite table)
static int lag_rmax(int d, bool dbl) {
    switch (d) {
        case 1:
        case 2: return 8;
        case 3: return dbl ? 4 : 6;
        case 4: return 4;
        default: return -1;
    }
}

int lag_table_size(int d, int R, bool dbl) {
    if (R < 0 || R > lag_rmax(d, dbl)) return 0;
    const int Re = (R + 1) & ~1;   // even instantiations
    long long c = 1;
    for (int i = 1; i <= d; ++i) c = c * (Re + i) / i;
    return (int)c;
}

template <typename real, int D, int R>
static cudaError_t lag_go(const LagItem<real>* items, const LagTile* tiles, int ntiles, const real* wpool,
                          double* partial, int grid, cudaStream_t st) {
    k_lag<real, D, R><<<grid, 256, 0, st>>>(items, tiles, ntiles, wpool, partial);
    return cudaGetLastError();
}

template <typename real, int D>
static cudaError_t lag_d(int R, const LagItem<real>* items, const LagTile* tiles, int ntiles, const real* wpool,
                         double* partial, int grid, cudaStream_t st) {
    constexpr bool dbl = sizeof(real) == 8;
    const int Re = (R + 1) & ~1;
    if (Re > lag_rmax(D, dbl)) return cudaErrorNotSupported;
    switch (Re) {
        case 0: return lag_go<real, D, 0>(items, tiles, ntiles, wpool, partial, grid, st);
        case 2: return lag_go<real, D, 2>(items, tiles, ntiles, wpool, partial, grid, st);
        case 4: return lag_go<real, D, 4>(items, tiles, ntiles, wpool, partial, grid, st);
        case 6:
            if constexpr (D <= 2 || (D == 3 && !dbl)) return lag_go<real, D, 6>(items, tiles, ntiles, wpool, partial, grid, st);
            return cudaErrorNotSupported;
        case 8:
            if constexpr (D <= 2) return lag_go<real, D, 8>(items, tiles, ntiles, wpool, partial, grid, st);
            return cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
    }
}

template <typename real>
cudaError_t launch_lag(int d, int R, const LagItem<real>* items, const LagTile* tiles, int ntiles, const real* wpool,
                       double* partial, int grid, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    switch (d) {
        case 1: return lag_d<real, 1>(R, items, tiles, ntiles, wpool, partial, grid, st);
        case 2: return lag_d<real, 2>(R, items, tiles, ntiles, wpool, partial, grid, st);
        case 3: return lag_d<real, 3>(R, items, tiles, ntiles, wpool, partial, grid, st);
        case 4: return lag_d<real, 4>(R, items, tiles, ntiles, wpool, partial, grid, st);
        default: return cudaErrorNotSupported;
    }
}

template <typename real>
cudaError_t launch_lag_reduce(const LagItem<real>* items, int nitems, const double* partial, double* out,
                              cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    k_lag_reduce<real><<<(nitems + 127) / 128, 128, 0, st>>>(items, nitems, partial, out);
    return cudaGetLastError();
}

template cudaError_t launch_lag<float>(int, int, const LagItem<float>*, const LagTile*, int, const float*, double*, int,
                                       cudaStream_t);
template cudaError_t launch_lag<double>(int, int, const LagItem<double>*, const LagTile*, int, const double*, double*,
                                        int, cudaStream_t);
template cudaError_t launch_lag_reduce<float>(const LagItem<float>*, int, const double*, double*, cudaStream_t);
template cudaError_t launch_lag_reduce<double>(const LagItem<double>*, int, const double*, double*, cudaStream_t);

}  // namespace kdefft
