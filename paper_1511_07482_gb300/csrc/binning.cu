// Step 1 of Sec. 4: binning of the sample onto the grid.
//
// Linear binning (the multilinear rule the paper takes from Wand 1994):
//   inside iff lo_k <= x_k <= hi_k on every axis (the grid range contains
//   the data); t_k = (x_k - lo_k) * (1 / delta_k) (FP64, each operation
//   rounded separately, no contraction; within two ulps of the quotient),
//   clamped to M_k - 1 because the rounding of delta_k can push a point at
//   hi_k just past it
//   l_k = floor(t_k), clamped to M_k - 2 on the upper edge; f_k = t_k - l_k
//   corner l + b receives prod_k (b_k ? f_k : 1 - f_k), product in axis order.
// Simple binning: weight 1 at l_k = floor(t_k + 1/2), with t_k the quotient
// (x_k - lo_k) / delta_k itself, so that the cells match the oracle's bit for
// bit.
//
// Grids that fit in shared memory are accumulated per block there (one
// privatised histogram per block, flushed with global atomics of the nonzero
// cells); larger grids use global atomics directly.
//
// FP32 counts are accumulated in 64-bit fixed point (each weight rounded to
// a multiple of 2^-K, K = 32 for samples below 2^31 points): integer sums do
// not depend on the order of the atomic additions, so the counts, and every
// objective value computed from them, are the same from run to run.  Their
// corner weights are FP32 products of the FP64 fractions rounded to FP32: a
// weight's relative error of a few 2^-24 matches the FP32 rounding of the
// count itself.  FP64 counts use FP64 weights and FP64 atomics.
#include <type_traits>

#include "engine.cuh"

namespace kdefft {

// Linear binning locates a point with t = (x - lo) * (1 / delta): one FP64
// multiply instead of a division (FP64 is slow on this part).  t is within
// two ulps of the oracle's (x - lo) / delta, so a point moves to the next
// cell only within two ulps of a node, where its weight there is ~1e-16.
struct Recip {
    double v[MAXD];
};

__device__ __forceinline__ bool locate(const double* __restrict__ x, const GridDesc& g, const Recip& inv, long long* l,
                                       double* f, long long* base) {
    long long b = 0;
    for (int k = 0; k < g.d; ++k) {
        if (!(x[k] >= g.lo[k] && x[k] <= g.hi[k])) return false;   // NaN fails too
        const double top = (double)(g.M[k] - 1);
        const double t = fmin(__dmul_rn(__dsub_rn(x[k], g.lo[k]), inv.v[k]), top);
        double lk = floor(t);
        if (lk >= top) lk = top - 1.0;
        f[k] = __dsub_rn(t, lk);
        l[k] = (long long)lk;
        b = b * g.M[k] + l[k];
    }
    *base = b;
    return true;
}

// Fixed-point weight of a corner (units of 2^-K, qscale = 2^K) from FP32
// factors: the location t, l, f stays FP64 as above, but the corner product
// only feeds an FP32 count, and a few FP32 roundings of the weight stay at
// the level of that count's own rounding (FP64 arithmetic is slow here).
__device__ __forceinline__ unsigned long long corner_fixed(int d, int c, const float* ff, const float* gg,
                                                           float qscale) {
    float w = 1.f;
    for (int k = 0; k < d; ++k) w *= ((c >> k) & 1) ? ff[k] : gg[k];
    return __float2ull_rn(w * qscale);
}

template <typename acc>
__global__ void __launch_bounds__(256) k_bin_linear(const double* __restrict__ X, long long n, GridDesc g, Recip inv,
                                                    acc* __restrict__ counts, long long ncells,
                                                    unsigned long long* __restrict__ outside, int use_smem,
                                                    double qscale) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    acc* hist = reinterpret_cast<acc*>(smem_raw);
    if (use_smem) {
        for (long long c = threadIdx.x; c < ncells; c += blockDim.x) hist[c] = acc(0);
        __syncthreads();
    }
    long long stride[MAXD];
    {
        long long s = 1;
        for (int k = g.d - 1; k >= 0; --k) {
            stride[k] = s;
            s *= g.M[k];
        }
    }
    const int ncorner = 1 << g.d;
    constexpr bool fixed = std::is_same<acc, unsigned long long>::value;
    const float qs = (float)qscale;   // 2^K, exact
    unsigned long long nout = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double x[MAXD], f[MAXD];
        long long l[MAXD], base;
        for (int k = 0; k < g.d; ++k) x[k] = X[i * g.d + k];
        if (!locate(x, g, inv, l, f, &base)) {
            ++nout;
            continue;
        }
        float ff[MAXD], gg[MAXD];
        if constexpr (fixed)
            for (int k = 0; k < g.d; ++k) {
                ff[k] = (float)f[k];
                gg[k] = 1.f - ff[k];
            }
        for (int b = 0; b < ncorner; ++b) {
            long long idx = base;
            for (int k = 0; k < g.d; ++k) idx += ((b >> k) & 1) * stride[k];
            acc* dst = use_smem ? hist + idx : counts + idx;
            if constexpr (fixed) {
                atomicAdd(dst, corner_fixed(g.d, b, ff, gg, qs));
            } else {
                double w = 1.0;
                for (int k = 0; k < g.d; ++k) w = __dmul_rn(w, ((b >> k) & 1) ? f[k] : __dsub_rn(1.0, f[k]));
                atomicAdd(dst, w);
            }
        }
    }
    if (nout) atomicAdd(outside, nout);
    if (use_smem) {
        __syncthreads();
        for (long long c = threadIdx.x; c < ncells; c += blockDim.x) {
            const acc v = hist[c];
            if (v != acc(0)) atomicAdd(counts + c, v);
        }
    }
}

__global__ void __launch_bounds__(256) k_bin_simple(const double* __restrict__ X, long long n, GridDesc g,
                                                    int* __restrict__ counts, unsigned long long* __restrict__ outside) {
    unsigned long long nout = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        long long idx = 0;
        bool ok = true;
        for (int k = 0; k < g.d; ++k) {
            const double x = X[i * g.d + k];
            if (!(x >= g.lo[k] && x <= g.hi[k])) {
                ok = false;
                break;
            }
            const double t = fmin(__ddiv_rn(__dsub_rn(x, g.lo[k]), g.delta[k]), (double)(g.M[k] - 1));
            const long long lk = (long long)floor(__dadd_rn(t, 0.5));
            idx = idx * g.M[k] + lk;
        }
        if (!ok) {
            ++nout;
            continue;
        }
        atomicAdd(counts + idx, 1);
    }
    if (nout) atomicAdd(outside, nout);
}

__global__ void k_f32_to_f64(const float* __restrict__ src, double* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

cudaError_t launch_f32_to_f64(const float* src, double* dst, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    k_f32_to_f64<<<(int)b, 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

__global__ void k_fix_to_f32(const unsigned long long* __restrict__ src, float* __restrict__ dst, long long n,
                             double unit) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (float)((double)src[i] * unit);
}

cudaError_t launch_fix_to_f32(const unsigned long long* src, float* dst, long long n, double unit, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    k_fix_to_f32<<<(int)b, 256, 0, st>>>(src, dst, n, unit);
    return cudaGetLastError();
}

template <typename real>
__global__ void k_int_to_real(const int* __restrict__ src, real* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (real)src[i];
}

static int blocks_for(long long n, int nsm, int per_sm) {
    long long b = (n + 255) / 256;
    const long long cap = (long long)nsm * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename acc>
cudaError_t launch_bin_linear(const double* X, long long n, const GridDesc& g, acc* counts, long long ncells,
                              unsigned long long* outside, double qscale, int nsm, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const size_t hist_bytes = sizeof(acc) * (size_t)ncells;
    const int use_smem = hist_bytes <= 96 * 1024;
    size_t sm = 0;
    int grid;
    if (use_smem) {
        sm = hist_bytes;   // within the 96 KB set once by prepare_binning (no attribute call here: graph capture)
        grid = blocks_for(n, nsm, 2);
    } else {
        grid = blocks_for(n, nsm, 8);
    }
    Recip inv{};
    for (int k = 0; k < g.d; ++k) inv.v[k] = 1.0 / g.delta[k];
    k_bin_linear<acc><<<grid, 256, sm, st>>>(X, n, g, inv, counts, ncells, outside, use_smem, qscale);
    return cudaGetLastError();
}

cudaError_t launch_bin_simple(const double* X, long long n, const GridDesc& g, int* counts, long long ncells,
                              unsigned long long* outside, int nsm, cudaStream_t st) {
    (void)ncells;
    if (n <= 0) return cudaSuccess;
    k_bin_simple<<<blocks_for(n, nsm, 8), 256, 0, st>>>(X, n, g, counts, outside);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_int_to_real(const int* src, real* dst, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    k_int_to_real<real><<<(int)b, 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

// Sample covariance for the normal-scale start point, in one pass: FP64
// block sums of x - s and (x - s)(x - s)^T
// with a fixed shift s inside the data (the grid's centre), from which
// cov = (S2 - S1 S1^T / n) / (n - 1); with s near the mean the subtraction
// loses little.  out: per block d + d^2 values.
__global__ void __launch_bounds__(256) k_moments_shifted(const double* __restrict__ X, long long n, int d, Shift sh,
                                                         double* __restrict__ out) {
    double acc[MAXD + MAXD * MAXD];
    const int nv = d + d * d;
    for (int v = 0; v < nv; ++v) acc[v] = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double x[MAXD];
        for (int k = 0; k < d; ++k) x[k] = X[i * d + k] - sh.s[k];
        for (int k = 0; k < d; ++k) acc[k] += x[k];
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) acc[d + a * d + b] += x[a] * x[b];
    }
    __shared__ double red[8][MAXD + MAXD * MAXD];
    for (int v = 0; v < nv; ++v) {
        double t = acc[v];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][v] = t;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
        out[(size_t)blockIdx.x * nv + threadIdx.x] = t;   // block partial; summed in block order by the host
    }
}

cudaError_t launch_moments_shifted(const double* X, long long n, int d, const Shift& sh, double* out, int nsm,
                                   cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_moments_shifted<<<moments_blocks(n, nsm), 256, 0, st>>>(X, n, d, sh, out);
    return cudaGetLastError();
}

int moments_blocks(long long n, int nsm) { return blocks_for(n, nsm, 2); }


// ------------------------------------------------------------ batched binning
__device__ __forceinline__ int bin_job_of(const BinJob* __restrict__ jobs, int n, long long b) {
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

constexpr int kBinPtsPerBlock = 256 * 8;
constexpr int kCellsPerBlock = 256 * 4;

__global__ void __launch_bounds__(256) k_bin_many(const BinJob* __restrict__ jobs, int njobs, int phase,
                                                  double qscale) {
    const BinJob& jb = jobs[bin_job_of(jobs, njobs, blockIdx.x)];
    const long long b = (long long)blockIdx.x - jb.blk0;
    const GridDesc& g = jb.g;
    const int d = g.d;
    if (phase == 0) {
        long long stride[MAXD];
        {
            long long s = 1;
            for (int k = d - 1; k >= 0; --k) {
                stride[k] = s;
                s *= g.M[k];
            }
        }
        const int ncorner = 1 << d;
        Recip inv{};   // the same correctly rounded reciprocals as launch_bin_linear's
        for (int k = 0; k < d; ++k) inv.v[k] = __drcp_rn(g.delta[k]);
        unsigned long long nout = 0;
        const long long i0 = b * kBinPtsPerBlock;
        const long long i1 = i0 + kBinPtsPerBlock < jb.n ? i0 + kBinPtsPerBlock : jb.n;
        for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            double x[MAXD], f[MAXD];
            long long l[MAXD], base;
            for (int k = 0; k < d; ++k) x[k] = jb.X[i * d + k];
            if (!locate(x, g, inv, l, f, &base)) {
                ++nout;
                continue;
            }
            float ff[MAXD], gg[MAXD];
            for (int k = 0; k < d; ++k) {
                ff[k] = (float)f[k];
                gg[k] = 1.f - ff[k];
            }
            const float qs = (float)qscale;
            for (int c = 0; c < ncorner; ++c) {
                long long idx = base;
                for (int k = 0; k < d; ++k) idx += ((c >> k) & 1) * stride[k];
                atomicAdd(jb.fix + idx, corner_fixed(d, c, ff, gg, qs));
            }
        }
        if (nout) atomicAdd(jb.outside, nout);
    } else if (phase == 1) {
        const double unit = 1.0 / qscale;
        const long long c0 = b * kCellsPerBlock;
        const long long c1 = c0 + kCellsPerBlock < jb.ncells ? c0 + kCellsPerBlock : jb.ncells;
        for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) jb.counts[c] = (float)((double)jb.fix[c] * unit);
    } else {
        // covariance in one pass, shifted by the grid's centre (as
        // k_moments_shifted): block b of mblk takes the points i = b, b + mblk,
        // ... in steps of blockDim
        const int nv = d + d * d;
        double acc[MAXD + MAXD * MAXD];
        for (int v = 0; v < nv; ++v) acc[v] = 0.0;
        for (long long i = b * blockDim.x + threadIdx.x; i < jb.n; i += (long long)jb.mblk * blockDim.x) {
            double x[MAXD];
            for (int k = 0; k < d; ++k) x[k] = jb.X[i * d + k] - jb.shift[k];
            for (int k = 0; k < d; ++k) acc[k] += x[k];
            for (int a = 0; a < d; ++a)
                for (int c = 0; c < d; ++c) acc[d + a * d + c] += x[a] * x[c];
        }
        __shared__ double red[8][MAXD + MAXD * MAXD];
        for (int v = 0; v < nv; ++v) {
            double t = acc[v];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][v] = t;
        }
        __syncthreads();
        if (threadIdx.x < nv) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
            jb.part[b * nv + threadIdx.x] = t;
        }
    }
}

cudaError_t launch_bin_many(BinJob* jobs_h, BinJob* jobs_d, int n, int phase, double qscale, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long blocks = 0;
    for (int k = 0; k < n; ++k) {
        BinJob& jb = jobs_h[k];
        jb.blk0 = blocks;
        if (phase == 0)
            blocks += (jb.n + kBinPtsPerBlock - 1) / kBinPtsPerBlock;
        else if (phase == 1)
            blocks += (jb.ncells + kCellsPerBlock - 1) / kCellsPerBlock;
        else
            blocks += jb.mblk;
    }
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyAsync(jobs_d, jobs_h, sizeof(BinJob) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    k_bin_many<<<(unsigned)blocks, 256, 0, st>>>(jobs_d, n, phase, qscale);
    return cudaGetLastError();
}

cudaError_t prepare_binning() {
    cudaError_t e = cudaFuncSetAttribute(k_bin_linear<unsigned long long>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_bin_linear<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
}

template cudaError_t launch_bin_linear<unsigned long long>(const double*, long long, const GridDesc&,
                                                           unsigned long long*, long long, unsigned long long*, double,
                                                           int, cudaStream_t);
template cudaError_t launch_bin_linear<double>(const double*, long long, const GridDesc&, double*, long long,
                                               unsigned long long*, double, int, cudaStream_t);
template cudaError_t launch_int_to_real<float>(const int*, float*, long long, cudaStream_t);
template cudaError_t launch_int_to_real<double>(const int*, double*, long long, cudaStream_t);

}  // namespace kdefft
