// Device helpers shared by the kernel files (engine.cu, lag.cu): compensated
// FP32 accumulation, block reductions to FP64, and the compile-time
// multivariate Hermite recurrence.  Internal; not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

namespace kdefft {

// ---- accumulation.  FP64 arithmetic is slow on this part, so FP32 sums
// carry an error term (two-sum / double-float): the pair (h, l) holds the
// sum to about u^2 relative, and it becomes FP64 once per block.
struct DFloat {
    float h, l;
};
__device__ __forceinline__ DFloat df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DFloat df_add(DFloat a, DFloat b) {
    const DFloat s = df_two_sum(a.h, b.h);
    const float e = s.l + (a.l + b.l);
    const float h = s.h + e;
    return {h, e - (h - s.h)};
}
// a b for FP32 a, b as an unevaluated pair: exact (the fused multiply-add
// gives the product's rounding error)
__device__ __forceinline__ DFloat df_prod(float a, float b) {
    const float p = a * b;
    return DFloat{p, fmaf(a, b, -p)};
}
// (a.h + a.l)(b.h + b.l) to a few units of 2^-44 relative
__device__ __forceinline__ DFloat df_mul(DFloat a, DFloat b) {
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)));
    const float s = p + e;
    return DFloat{s, e - (s - p)};
}
// (a.h + a.l) b for an FP32 b
__device__ __forceinline__ DFloat df_mulf(DFloat a, float b) {
    const float p = a.h * b;
    const float e = fmaf(a.l, b, fmaf(a.h, b, -p));
    const float s = p + e;
    return DFloat{s, e - (s - p)};
}
__device__ __forceinline__ void df_acc(DFloat& a, float x) {
    const DFloat s = df_two_sum(a.h, x);
    const float e = s.l + a.l;
    a.h = s.h + e;
    a.l = e - (a.h - s.h);
}

// ---- an FP32 pair x = h + l with |l| <= ulp(h) / 2 as an arithmetic type
// (about 44 significant bits), so that templated transforms can run on the
// FP32 pipes where FP64 would be slow.  Sums renormalise through two-sum,
// products through the fused multiply-add's exact rounding error; both keep
// the error a few units of 2^-44 of the operands' magnitudes, which is what
// a transform's error bound needs.  Constants come from double literals,
// split at compile time.
struct dflt {
    float h, l;
    __host__ __device__ constexpr dflt() : h(0.f), l(0.f) {}
    __host__ __device__ constexpr dflt(float a, float b) : h(a), l(b) {}
    __host__ __device__ constexpr explicit dflt(double v) : h((float)v), l((float)(v - (double)(float)v)) {}
};
__device__ __forceinline__ dflt operator+(dflt a, dflt b) {
    const float s = a.h + b.h;
    const float bb = s - a.h;
    const float e = ((a.h - (s - bb)) + (b.h - bb)) + (a.l + b.l);
    const float h = s + e;
    return dflt(h, e - (h - s));
}
__device__ __forceinline__ dflt operator-(dflt a) { return dflt(-a.h, -a.l); }
__device__ __forceinline__ dflt operator-(dflt a, dflt b) { return a + (-b); }
__device__ __forceinline__ dflt operator*(dflt a, dflt b) {
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)));
    const float h = p + e;
    return dflt(h, e - (h - p));
}
__device__ __forceinline__ double to_double(dflt a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ double to_double(double a) { return a; }
// complex FP32 pair: the layout and size of double2
struct dcplx {
    dflt x, y;
};

// per-thread accumulator of the spectral sums: DFloat in FP32 mode, double in FP64 mode
template <typename real>
struct SumAcc;
template <>
struct SumAcc<float> {
    DFloat a{0.f, 0.f}, b{0.f, 0.f};
    __device__ __forceinline__ void add(float x, float y) {
        df_acc(a, x);
        df_acc(b, y);
    }
};
template <>
struct SumAcc<double> {
    double a = 0.0, b = 0.0;
    __device__ __forceinline__ void add(double x, double y) {
        a += x;
        b += y;
    }
};

// block sum of a SumAcc; thread 0 receives the two totals as doubles.
// Contains __syncthreads (call from uniform control flow).
__device__ __forceinline__ void block_reduce_acc(const SumAcc<float>& s, double* out2) {
    __shared__ DFloat red[2][32];
    DFloat a = s.a, b = s.b;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DFloat ta{__shfl_down_sync(0xffffffffu, a.h, o), __shfl_down_sync(0xffffffffu, a.l, o)};
        DFloat tb{__shfl_down_sync(0xffffffffu, b.h, o), __shfl_down_sync(0xffffffffu, b.l, o)};
        a = df_add(a, ta);
        b = df_add(b, tb);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = a;
        red[1][w] = b;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        a = (l < nw) ? red[0][l] : DFloat{0.f, 0.f};
        b = (l < nw) ? red[1][l] : DFloat{0.f, 0.f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            DFloat ta{__shfl_down_sync(0xffffffffu, a.h, o), __shfl_down_sync(0xffffffffu, a.l, o)};
            DFloat tb{__shfl_down_sync(0xffffffffu, b.h, o), __shfl_down_sync(0xffffffffu, b.l, o)};
            a = df_add(a, ta);
            b = df_add(b, tb);
        }
        if (l == 0) {
            out2[0] = (double)a.h + (double)a.l;
            out2[1] = (double)b.h + (double)b.l;
        }
    }
    __syncthreads();
}
template <typename real>
__device__ void block_reduce2(double a, double b, double* out2) {
    __shared__ double red[2][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = a;
        red[1][w] = b;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        a = (l < nw) ? red[0][l] : 0.0;
        b = (l < nw) ? red[1][l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (l == 0) {
            out2[0] = a;
            out2[1] = b;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void block_reduce_acc(const SumAcc<double>& s, double* out2) {
    block_reduce2<double>(s.a, s.b, out2);
}

// ------------------------------------------------------------ compile-time Hermite recurrence
// The same graded enumeration and recurrence as the constant-memory table,
// generated at compile time for fixed (D, R) so that the polynomials live in
// registers and every index is a constant.
constexpr int cx_binom(int n, int k) {
    long long c = 1;
    for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
    return (int)c;
}

template <int D, int R>
struct HTab {
    static constexpr int N = cx_binom(D + R, D);
    int al[N][D];
    int piv[N];
    int par[N];
    int nred[N];
    int rj[N][D];
    int rc[N][D];
    int ridx[N][D];
    constexpr int index_of(const int* a) const {
        for (int t = 0; t < N; ++t) {
            bool eq = true;
            for (int k = 0; k < D; ++k) eq = eq && (al[t][k] == a[k]);
            if (eq) return t;
        }
        return -1;
    }
    constexpr HTab() : al(), piv(), par(), nred(), rj(), rc(), ridx() {
        int n = 0;
        for (int o = 0; o <= R; ++o) {
            // all alpha with |alpha| = o, alpha_0 descending, then alpha_1, ...
            int a[D] = {};
            a[0] = o;
            for (;;) {
                int used = 0;
                for (int k = 0; k < D - 1; ++k) used += a[k];
                a[D - 1] = o - used;
                if (a[D - 1] >= 0) {
                    for (int k = 0; k < D; ++k) al[n][k] = a[k];
                    ++n;
                }
                int k = D - 2;
                for (; k >= 0; --k)
                    if (a[k] > 0) break;
                if (k < 0) break;
                a[k]--;
                int pre = 0;
                for (int m = 0; m <= k; ++m) pre += a[m];
                if (k + 1 <= D - 2) {
                    a[k + 1] = o - pre;
                    for (int m = k + 2; m <= D - 2; ++m) a[m] = 0;
                }
            }
        }
        for (int t = 1; t < N; ++t) {
            int p = 0;
            while (al[t][p] == 0) ++p;
            int beta[D] = {};
            for (int k = 0; k < D; ++k) beta[k] = al[t][k];
            beta[p] -= 1;
            piv[t] = p;
            par[t] = index_of(beta);
            for (int j = 0; j < D; ++j)
                if (beta[j] > 0) {
                    int g[D] = {};
                    for (int k = 0; k < D; ++k) g[k] = beta[k];
                    g[j] -= 1;
                    rj[t][nred[t]] = j;
                    rc[t][nred[t]] = beta[j];
                    ridx[t][nred[t]] = index_of(g);
                    nred[t]++;
                }
        }
    }
};

}  // namespace kdefft
