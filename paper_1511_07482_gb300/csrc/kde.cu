// The kernel density estimate on the grid and the cross term of the
// integrated squared error against a normal mixture, for the binned sample.
//
//   kde_grid  f_hat(g) = n^-1 sum_{|l_k| <= L_k} c_{g - l} K_H(delta (.) l) at
//             every grid node g (the binned estimator, the convolution that
//             Eqs. 19-24 evaluate through the FFT, truncated as in Eq. 26),
//             one thread per node, the stencil K_H(delta (.) l) from a table,
//             compensated FP32 sums written as FP64.
//   mix_dot   sum_g c_g sum_m w_m phi_{S_m}(x_g - mu_m) (FP64), one FP64
//             partial per block, summed in block order by the host.
#include "devutil.cuh"
#include "engine.cuh"

namespace kdefft {

__global__ void __launch_bounds__(256) k_kde_grid(const float* __restrict__ counts, KdeDesc g,
                                                  const float* __restrict__ ktab, double* __restrict__ out) {
    const int d = g.d;
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncells;
         cell += (long long)gridDim.x * blockDim.x) {
        int idx[MAXD] = {0, 0, 0, 0};
        {
            long long r = cell;
            for (int k = d - 1; k >= 0; --k) {
                idx[k] = (int)(r % g.M[k]);
                r /= g.M[k];
            }
        }
        int l[MAXD] = {0, 0, 0, 0};
        for (int k = 0; k < d; ++k) l[k] = -g.L[k];
        DFloat acc{0.f, 0.f};
        for (long long s = 0; s < g.nstencil; ++s) {
            long long src = 0;
            bool in = true;
            for (int k = 0; k < d; ++k) {
                const int q = idx[k] - l[k];
                in = in && q >= 0 && q < g.M[k];
                src = src * g.M[k] + q;
            }
            if (in) {
                const float cv = counts[src];
                if (cv != 0.f) df_acc(acc, cv * ktab[s]);
            }
            for (int k = d - 1; k >= 0; --k) {   // next stencil point, last axis fastest
                if (++l[k] <= g.L[k]) break;
                l[k] = -g.L[k];
            }
        }
        out[cell] = ((double)acc.h + (double)acc.l) * g.inv_n;
    }
}

cudaError_t launch_kde_grid(const float* counts, const KdeDesc& g, const float* ktab, double* out, int nsm,
                            cudaStream_t st) {
    if (g.ncells <= 0) return cudaSuccess;
    long long b = (g.ncells + 255) / 256;
    const long long cap = (long long)nsm * 8;
    if (b > cap) b = cap;
    k_kde_grid<<<(int)b, 256, 0, st>>>(counts, g, ktab, out);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_mix_dot(const float* __restrict__ counts, KdeDesc g,
                                                 const MixComp* __restrict__ comps, int ncomp,
                                                 double* __restrict__ partial) {
    const int d = g.d;
    double acc = 0.0;
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncells;
         cell += (long long)gridDim.x * blockDim.x) {
        const float cv = counts[cell];
        if (cv == 0.f) continue;
        double x[MAXD] = {0.0, 0.0, 0.0, 0.0};
        {
            long long r = cell;
            for (int k = d - 1; k >= 0; --k) {
                const int i = (int)(r % g.M[k]);
                r /= g.M[k];
                x[k] = g.lo[k] + g.delta[k] * (double)i;
            }
        }
        double f = 0.0;
        for (int m = 0; m < ncomp; ++m) {
            const MixComp& c = comps[m];
            double z[MAXD], q = 0.0;
            for (int k = 0; k < d; ++k) z[k] = x[k] - c.mu[k];
            for (int a = 0; a < d; ++a) {
                double t = 0.0;
                for (int b = 0; b < d; ++b) t += c.lam[a * MAXD + b] * z[b];
                q += z[a] * t;
            }
            f += c.w * c.nrm * exp(-0.5 * q);
        }
        acc += (double)cv * f;
    }
    double out2[2];
    block_reduce2<double>(acc, 0.0, out2);
    if (threadIdx.x == 0) partial[blockIdx.x] = out2[0];
}

cudaError_t launch_mix_dot(const float* counts, const KdeDesc& g, const MixComp* comps, int ncomp, double* partial,
                           int nblocks, cudaStream_t st) {
    k_mix_dot<<<nblocks, 256, 0, st>>>(counts, g, comps, ncomp, partial);
    return cudaGetLastError();
}

}  // namespace kdefft
