// Lag-domain evaluation of the binned functionals (Eq. 25 with the sum over
// the lag done first) against the count autocorrelation (whose passes run
// in engine.cu with the other transforms).
//
//   lag      per work item (two kernels of the same covariances and
//            support, as in the FFT path), sum over the half lag box of
//            w_j k_j a_j, w_j in {0, 1, 2}; kernels from the compile-time
//            Hermite recurrence; compensated FP32 sums with one FP64
//            partial per tile, or FP64 sums with one partial per warp slice
//            of a tile.
//   lag_sum  fixed-order sum of each item's tile partials, times n^-2, for
//            the items of every batch of a run in one launch.
#include <algorithm>

#include "devutil.cuh"
#include "engine.cuh"

namespace kdefft {

// floor(n / v) for a 32-bit n from the invariant divisor's multiplier m and
// shifts (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994, unsigned case): t = mulhi(m, n), then
// (t + ((n - t) >> s1)) >> s2; exact for every 32-bit n.
__device__ __forceinline__ uint32_t inv_div(uint32_t n, uint32_t m, int sh) {
    const uint32_t t = __umulhi(m, n);
    return (t + ((n - t) >> (sh & 0xff))) >> (sh >> 8);
}

// ------------------------------------------------------------ lag evaluation
// tiles [t0, t0 + ntiles) of the batch's tile list.  FP32: a tile per CTA
// (256 threads, thread t takes the tile's points t, t + 256, ...), one
// partial pair per tile.  FP64: a tile's 256 points are 8 warp slices of one
// point per thread; a CTA of blockDim threads takes blockDim / 32 slices of
// a tile, and each warp writes its slice's pair (partial holds kLagSlices
// pairs per tile).  A thread's points and a warp's shuffle tree are the same
// for every block size, so the partials are too.
template <typename real, int D, int R>
__device__ __forceinline__ void lag_tiles(const LagItem<real>* __restrict__ items, const LagTile* __restrict__ tiles,
                                          int t0, int ntiles, const real* __restrict__ wpool,
                                          double* __restrict__ partial) {
    constexpr bool dbl = sizeof(real) == 8;
    constexpr HTab<D, R> ht{};
    constexpr int N = HTab<D, R>::N;
    __shared__ real Ws[2][MAXSIG][N];
    __shared__ LagItem<real> it;
    const int wpc = (int)(blockDim.x >> 5);               // warps (FP64: slices) per CTA
    const int per = dbl ? kLagSlices / wpc : 1;           // CTAs per tile
    const long long nunits = (long long)ntiles * per;
    for (long long u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int tix = t0 + (int)(u / per);
        const int s0 = dbl ? (int)(u % per) * wpc : 0;   // first slice of this CTA
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
        const int vstride = dbl ? 32 * kLagSlices : (int)blockDim.x;
        for (long long f = tl.first + s0 * 32 + threadIdx.x; f < end; f += vstride) {
            // the flat index splits into (j_0, .., j_{d-1}) by exact 32-bit
            // divisions (the engine takes half boxes below 2^32 points)
            int j[D];
            uint32_t g = (uint32_t)f;
#pragma unroll
            for (int k = 0; k < D - 1; ++k) {
                const uint32_t w = (k == 0) ? (uint32_t)n0 : (uint32_t)(2 * it.L[k] + 1);
                const uint32_t qv = inv_div(g, it.qm[k], it.qs[k]);
                j[k] = (int)(g - qv * w) - (k == 0 ? 0 : it.L[k]);
                g = qv;
            }
            j[D - 1] = (int)g - (D == 1 ? 0 : it.L[D - 1]);
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
        if constexpr (dbl) {
            double a = acc.a, b = acc.b;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_down_sync(0xffffffffu, a, o);
                b += __shfl_down_sync(0xffffffffu, b, o);
            }
            if ((threadIdx.x & 31) == 0) {
                const long long slot = (long long)tix * kLagSlices + s0 + (threadIdx.x >> 5);
                partial[2 * slot] = a;
                partial[2 * slot + 1] = b;
            }
        } else {
            double out2[2];
            block_reduce_acc(acc, out2);
            if (threadIdx.x == 0) {
                partial[2 * (long long)tix] = out2[0];
                partial[2 * (long long)tix + 1] = out2[1];
            }
        }
    }
}

template <typename real, int D, int R>
__global__ void __launch_bounds__(256) k_lag(const LagItem<real>* __restrict__ items, const LagTile* __restrict__ tiles,
                                             int t0, int ntiles, const real* __restrict__ wpool,
                                             double* __restrict__ partial) {
    lag_tiles<real, D, R>(items, tiles, t0, ntiles, wpool, partial);
}

// The same, held to three CTAs per SM (taken for the 3-D fourth-order FP32
// kernel: 80 registers and a 20-byte spill, where the compiler's own choice
// of 98 registers leaves two CTAs per SM; psi_4 of 256 bandwidths on a 128^3
// grid measured 192 against 221 us per launch.  The same cap on the 4-D
// kernel spilled 268 bytes and measured 64 against 54 us, so the others keep
// the compiler's choice.)
template <typename real, int D, int R>
__global__ void __launch_bounds__(256, 3) k_lag_occ3(const LagItem<real>* __restrict__ items,
                                                     const LagTile* __restrict__ tiles, int t0, int ntiles,
                                                     const real* __restrict__ wpool, double* __restrict__ partial) {
    lag_tiles<real, D, R>(items, tiles, t0, ntiles, wpool, partial);
}

// A FP64 tile's partial from its kLagSlices slice pairs (c = 0, 1): the
// order of a shuffle-down tree over the eight values (the block reduction
// these slices replace).
static_assert(kLagSlices == 8, "the combining order below is written for eight slices");
__device__ __forceinline__ double slices_sum(const double* __restrict__ p, int c) {
    return ((p[0 + c] + p[8 + c]) + (p[4 + c] + p[12 + c])) + ((p[2 + c] + p[10 + c]) + (p[6 + c] + p[14 + c]));
}

// One warp per item (of every batch of a run): lane l sums the item's tile
// partials l, l + 32, ... in order (a FP64 tile's from its slices first),
// then a fixed shuffle tree; times n^-2.
__global__ void __launch_bounds__(256) k_lag_sum(const LagSum* __restrict__ sums, int nitems,
                                                 const double* __restrict__ partial, double* __restrict__ out) {
    const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= nitems) return;   // whole warps leave together
    const LagSum sm = sums[i];
    double a = 0.0, b = 0.0;
    for (int t = lane; t < sm.ntile; t += 32) {
        const double* p = partial + 2 * (sm.tile0 + (long long)t * sm.nslice);
        if (sm.nslice == kLagSlices) {
            a += slices_sum(p, 0);
            b += slices_sum(p, 1);
        } else {
            a += p[0];
            b += p[1];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        out[2 * (long long)i] = a * sm.scale;
        out[2 * (long long)i + 1] = b * sm.scale;
    }
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
static cudaError_t lag_go(const LagJob<real>& j, cudaStream_t st) {
    if constexpr (sizeof(real) == 4 && D == 3 && R == 4)
        k_lag_occ3<real, D, R><<<j.grid, j.block, 0, st>>>(j.items, j.tiles, j.t0, j.ntiles, j.wpool, j.partial);
    else
        k_lag<real, D, R><<<j.grid, j.block, 0, st>>>(j.items, j.tiles, j.t0, j.ntiles, j.wpool, j.partial);
    return cudaGetLastError();
}

template <typename real, int D>
static cudaError_t lag_d(int R, const LagJob<real>& j, cudaStream_t st) {
    constexpr bool dbl = sizeof(real) == 8;
    const int Re = (R + 1) & ~1;
    if (Re > lag_rmax(D, dbl)) return cudaErrorNotSupported;
    switch (Re) {
        case 0: return lag_go<real, D, 0>(j, st);
        case 2: return lag_go<real, D, 2>(j, st);
        case 4: return lag_go<real, D, 4>(j, st);
        case 6:
            if constexpr (D <= 2 || (D == 3 && !dbl)) return lag_go<real, D, 6>(j, st);
            return cudaErrorNotSupported;
        case 8:
            if constexpr (D <= 2) return lag_go<real, D, 8>(j, st);
            return cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
    }
}

template <typename real>
cudaError_t launch_lag(int d, int R, const LagJob<real>& j, cudaStream_t st) {
    if (j.ntiles <= 0) return cudaSuccess;
    if (j.grid < 1) return cudaErrorInvalidValue;
    const bool slices_ok = sizeof(real) == 8 && (j.block == 32 || j.block == 64 || j.block == 128);
    if (j.block != 256 && !slices_ok) return cudaErrorInvalidValue;
    switch (d) {
        case 1: return lag_d<real, 1>(R, j, st);
        case 2: return lag_d<real, 2>(R, j, st);
        case 3: return lag_d<real, 3>(R, j, st);
        case 4: return lag_d<real, 4>(R, j, st);
        default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_lag_sum(const LagSum* sums, int nitems, const double* partial, double* out, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const long long threads = 32LL * nitems;
    k_lag_sum<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(sums, nitems, partial, out);
    return cudaGetLastError();
}

template cudaError_t launch_lag<float>(int, int, const LagJob<float>&, cudaStream_t);
template cudaError_t launch_lag<double>(int, int, const LagJob<double>&, cudaStream_t);

}  // namespace kdefft
