// Device kernels of the per-bandwidth hot path (Sec. 4 steps 2-4, Sec. 5):
//
//   stage_a   generates the sampled kernel k_j = sum_m w_m d^alpha phi_{Sigma_m}(delta (.) j)
//             (Eq. 18 / Eq. 34, Gaussian partials via the multivariate Hermite
//             recurrence) for a batch of lines along the last axis, directly in
//             shared memory, and transforms them (first FFT pass of Eq. 22).
//             For counts items it loads the grid counts instead (C = F(c_zp)).
//   mid       one FFT pass along an interior axis (only the support lines of
//             the axes not yet transformed are present: pruned transform).
//   final     the FFT pass along axis 0 fused with the spectral multiply-and-
//             reduce: sum_w |C_w|^2 K_w (discrete Parseval form of Eqs. 22-24,
//             equal to n^2 prod(P) times Eq. 25 when P_k >= M_k + L_k), or, for
//             counts items, the spectrum |C_w|^2.
//   reduce    fixed-order FP64 sum of the per-tile partials, times n^-2/prod P.
//
// The 1-D transforms are mixed-radix (2, 3, 4, 5, 8) Stockham passes over
// lines held in shared memory (self-sorting, ping-pong buffers), twiddles
// exp(-2 pi i t/P) from an FP64-computed table staged in shared memory.
#include <cooperative_groups.h>

#include "engine.cuh"

namespace cg = cooperative_groups;

namespace kdefft {

__constant__ HEnt c_htab[HMAX * 4];
__constant__ int c_hoff[5];

cudaError_t upload_hermite_tables(const HEnt* tab, const int* offsets, int total) {
    cudaError_t e = cudaMemcpyToSymbol(c_htab, tab, sizeof(HEnt) * total);
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_hoff, offsets, sizeof(int) * 5);
}

// ------------------------------------------------------------ complex helpers
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) { return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
// multiply by -i
template <typename C>
__device__ __forceinline__ C cmi(C a) { return C{a.y, -a.x}; }

// ------------------------------------------------------------ small DFTs (forward, e^{-2 pi i nk/R})
template <typename C, int R>
struct Dft;

template <typename C>
struct Dft<C, 2> {
    __device__ __forceinline__ static void run(C* v) {
        C a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    }
};

template <typename C>
struct Dft<C, 3> {
    __device__ __forceinline__ static void run(C* v) {
        using R_ = decltype(v[0].x);
        const R_ s = R_(0.8660254037844386);   // sin(2 pi / 3)
        C t1 = cadd(v[1], v[2]);
        C t2 = csub(v[1], v[2]);
        C m = C{v[0].x - R_(0.5) * t1.x, v[0].y - R_(0.5) * t1.y};
        C r = C{s * t2.y, -s * t2.x};   // -i s t2
        v[0] = cadd(v[0], t1);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};

template <typename C>
struct Dft<C, 4> {
    __device__ __forceinline__ static void run(C* v) {
        C a = cadd(v[0], v[2]);
        C b = csub(v[0], v[2]);
        C c = cadd(v[1], v[3]);
        C e = cmi(csub(v[1], v[3]));
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, e);
        v[3] = csub(b, e);
    }
};

template <typename C>
struct Dft<C, 5> {
    __device__ __forceinline__ static void run(C* v) {
        using R_ = decltype(v[0].x);
        const R_ c1 = R_(0.30901699437494745);   // cos(2 pi/5)
        const R_ c2 = R_(-0.8090169943749473);   // cos(4 pi/5)
        const R_ s1 = R_(0.9510565162951535);    // sin(2 pi/5)
        const R_ s2 = R_(0.5877852522924732);    // sin(4 pi/5)
        C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        C x0 = v[0];
        C p1 = C{x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y};
        C p2 = C{x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y};
        // q1 = s1 b1 + s2 b2, q2 = s2 b1 - s1 b2; X1 = p1 - i q1, X2 = p2 - i q2
        C q1 = C{s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y};
        C q2 = C{s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y};
        v[0] = C{x0.x + a1.x + a2.x, x0.y + a1.y + a2.y};
        v[1] = cadd(p1, cmi(q1));
        v[4] = csub(p1, cmi(q1));
        v[2] = cadd(p2, cmi(q2));
        v[3] = csub(p2, cmi(q2));
    }
};

template <typename C>
struct Dft<C, 8> {
    __device__ __forceinline__ static void run(C* v) {
        using R_ = decltype(v[0].x);
        const R_ h = R_(0.7071067811865476);     // sqrt(1/2)
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Dft<C, 4>::run(e);
        Dft<C, 4>::run(o);
        // o_k *= exp(-2 pi i k / 8)
        o[1] = C{h * (o[1].x + o[1].y), h * (o[1].y - o[1].x)};
        o[2] = cmi(o[2]);
        o[3] = C{h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y)};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 4] = csub(e[k], o[k]);
        }
    }
};

// ---- composite radices: R = A B with A the smallest prime factor, done in
// registers as A-point DFTs over stride-B subsequences, twiddles
// w_R^{b k1}, then B-point DFTs (X[k1 + A k2]).  The twiddles are compile-time
// constants: cos and sin of 2 pi m / R from an exact octant reduction of the
// rational m / R and a Taylor series on [0, pi/4].
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double cx_sin_t(double x) {
    double t = x, s = x;
    for (int i = 1; i < 14; ++i) {
        t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
        s += t;
    }
    return s;
}
constexpr double cx_cos_t(double x) {
    double t = 1.0, s = 1.0;
    for (int i = 1; i < 14; ++i) {
        t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
        s += t;
    }
    return s;
}
// (cos, sin) of 2 pi m / R
struct CxCis {
    double c, s;
};
constexpr CxCis cx_cis(int m, int R) {
    m %= R;
    if (m < 0) m += R;
    const int q = (8 * m) / R;   // octant
    const double x = kTwoPi * (double)(8 * m - q * R) / (8.0 * R);        // in [0, pi/4)
    const double y = kTwoPi * (double)(R * (q + 1) - 8 * m) / (8.0 * R);  // pi/4 - x
    switch (q) {
        case 0: return {cx_cos_t(x), cx_sin_t(x)};
        case 1: return {cx_sin_t(y), cx_cos_t(y)};
        case 2: return {-cx_sin_t(x), cx_cos_t(x)};
        case 3: return {-cx_cos_t(y), cx_sin_t(y)};
        case 4: return {-cx_cos_t(x), -cx_sin_t(x)};
        case 5: return {-cx_sin_t(y), -cx_cos_t(y)};
        case 6: return {cx_sin_t(x), -cx_cos_t(x)};
        default: return {cx_cos_t(y), -cx_sin_t(y)};
    }
}
constexpr int cx_small_factor(int R) {
    for (int f = 2; f <= R; ++f)
        if (R % f == 0) return f;
    return R;
}
template <int R>
struct CxTw {
    double c[R];
    double s[R];
    constexpr CxTw() : c(), s() {
        for (int m = 0; m < R; ++m) {
            const CxCis z = cx_cis(m, R);
            c[m] = z.c;
            s[m] = z.s;
        }
    }
};

template <typename C, int R>
struct Dft {
    __device__ __forceinline__ static void run(C* v) {
        using R_ = decltype(v[0].x);
        constexpr int A = cx_small_factor(R);
        constexpr int B = R / A;
        constexpr CxTw<R> tw{};
        C u[R];
        // A-point DFTs over b-strided subsequences: u[b * A + k1]
#pragma unroll
        for (int b = 0; b < B; ++b) {
            C t[A];
#pragma unroll
            for (int a = 0; a < A; ++a) t[a] = v[B * a + b];
            Dft<C, A>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) {
                const int m = (b * k1) % R;
                if (m == 0) {
                    u[b * A + k1] = t[k1];
                } else {
                    // t * exp(-2 pi i m / R) = t * (cos - i sin)
                    const R_ cw = R_(tw.c[m]), sw = R_(tw.s[m]);
                    u[b * A + k1] = C{t[k1].x * cw + t[k1].y * sw, t[k1].y * cw - t[k1].x * sw};
                }
            }
        }
        // B-point DFTs over b for each k1: X[k1 + A k2]
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
            C t[B];
#pragma unroll
            for (int b = 0; b < B; ++b) t[b] = u[b * A + k1];
            Dft<C, B>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = t[k2];
        }
    }
};

// n / D for n < 2^20 and 2 <= D <= 4096 as a multiply-high with
// m = ceil(2^32 / D): the rounding error n (m D - 2^32) / 2^32 < n D / 2^32
// stays below 1/D of the fractional gap, so the quotient is exact.
__device__ __forceinline__ uint32_t magic_of(uint32_t D) { return 0xFFFFFFFFu / D + 1u; }

// Line buffers in shared memory carry one pad element after every 16
// complex values: logical index i lives at i + i/16.  Stockham stores with
// stride R (R = 2, 4, 8) then fall on distinct banks instead of 2..16-way
// conflicts; unit-stride accesses stay contiguous.
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_cap(int cap) { return cap + (cap >> 4) + 1; }
__device__ __forceinline__ uint32_t qdiv(uint32_t n, uint32_t m) { return __umulhi(n, m); }

// One radix-R Stockham pass over nl lines of length P (dense, stride P).
template <typename C, int R>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ src, C* __restrict__ dst, int nl, int P,
                                              int Ns, const C* __restrict__ tw) {
    const int Pr = P / R;
    const int total = nl * Pr;
    const int tws = P / (Ns * R);
    const uint32_t mPr = magic_of((uint32_t)max(Pr, 2));
    const uint32_t mNs = magic_of((uint32_t)max(Ns, 2));
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int line = (Pr == 1) ? t : (int)qdiv((uint32_t)t, mPr);
        const int j = t - line * Pr;
        const int lb = line * P;
        const int k = (Ns == 1) ? 0 : j - (int)qdiv((uint32_t)j, mNs) * Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[pad(lb + j + r * Pr)];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[r * k * tws]);
        }
        Dft<C, R>::run(v);
        const int base = lb + (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[pad(base + r * Ns)] = v[r];
    }
}

// Forward DFT of nl lines (length P) held in a; b is the other buffer.
// Returns the buffer holding the result.  Ends with __syncthreads().
template <typename C>
__device__ __forceinline__ C* smem_fft(C* a, C* b, int nl, const AxisPlan& ap, const C* tw) {
    __syncthreads();
    int Ns = 1;
    C* src = a;
    C* dst = b;
    for (int s = 0; s < ap.nst; ++s) {
        const int R = ap.radix[s];
        if constexpr (sizeof(C) == 16) {
            switch (R) {
                case 2: stockham_pass<C, 2>(src, dst, nl, ap.P, Ns, tw); break;
                case 3: stockham_pass<C, 3>(src, dst, nl, ap.P, Ns, tw); break;
                case 4: stockham_pass<C, 4>(src, dst, nl, ap.P, Ns, tw); break;
                case 5: stockham_pass<C, 5>(src, dst, nl, ap.P, Ns, tw); break;
                case 6: stockham_pass<C, 6>(src, dst, nl, ap.P, Ns, tw); break;
                case 8: stockham_pass<C, 8>(src, dst, nl, ap.P, Ns, tw); break;
                case 9: stockham_pass<C, 9>(src, dst, nl, ap.P, Ns, tw); break;
                case 10: stockham_pass<C, 10>(src, dst, nl, ap.P, Ns, tw); break;
                case 12: stockham_pass<C, 12>(src, dst, nl, ap.P, Ns, tw); break;
                case 15: stockham_pass<C, 15>(src, dst, nl, ap.P, Ns, tw); break;
                default: stockham_pass<C, 16>(src, dst, nl, ap.P, Ns, tw); break;
            }
        } else {
            switch (R) {
                case 2: stockham_pass<C, 2>(src, dst, nl, ap.P, Ns, tw); break;
                case 3: stockham_pass<C, 3>(src, dst, nl, ap.P, Ns, tw); break;
                case 4: stockham_pass<C, 4>(src, dst, nl, ap.P, Ns, tw); break;
                case 5: stockham_pass<C, 5>(src, dst, nl, ap.P, Ns, tw); break;
                case 6: stockham_pass<C, 6>(src, dst, nl, ap.P, Ns, tw); break;
                case 8: stockham_pass<C, 8>(src, dst, nl, ap.P, Ns, tw); break;
                case 9: stockham_pass<C, 9>(src, dst, nl, ap.P, Ns, tw); break;
                case 10: stockham_pass<C, 10>(src, dst, nl, ap.P, Ns, tw); break;
                case 12: stockham_pass<C, 12>(src, dst, nl, ap.P, Ns, tw); break;
                case 15: stockham_pass<C, 15>(src, dst, nl, ap.P, Ns, tw); break;
                case 16: stockham_pass<C, 16>(src, dst, nl, ap.P, Ns, tw); break;
                case 18: stockham_pass<C, 18>(src, dst, nl, ap.P, Ns, tw); break;
                case 20: stockham_pass<C, 20>(src, dst, nl, ap.P, Ns, tw); break;
                case 24: stockham_pass<C, 24>(src, dst, nl, ap.P, Ns, tw); break;
                case 25: stockham_pass<C, 25>(src, dst, nl, ap.P, Ns, tw); break;
                case 27: stockham_pass<C, 27>(src, dst, nl, ap.P, Ns, tw); break;
                case 30: stockham_pass<C, 30>(src, dst, nl, ap.P, Ns, tw); break;
                default: stockham_pass<C, 32>(src, dst, nl, ap.P, Ns, tw); break;
            }
        }
        Ns *= R;
        __syncthreads();
        C* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// asynchronous global -> shared copies of 4, 8 or 16 bytes (cp.async); all of
// a tile's loads are in flight together, completed by cp_async_wait_all()
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gmem_src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename C>
__device__ __forceinline__ void load_twiddles(C* tw, const C* pool, const AxisPlan& ap) {
    for (int t = threadIdx.x; t < ap.P; t += blockDim.x) tw[t] = pool[ap.tw_off + t];
}

// ------------------------------------------------------------ kernel values

// Value of the packed pair (grid A + i grid B) at lag vector j (d entries).
template <typename real>
__device__ __forceinline__ void kernel_pair(const Item<real>& it, const int* j, real& va, real& vb) {
    real x[MAXD];
    const int d = it.d;
#pragma unroll
    for (int k = 0; k < MAXD; ++k) x[k] = (k < d) ? (real)it.delta[k] * (real)j[k] : real(0);
    real He[MAXSIG][HMAX];
    real ex[MAXSIG];
    const int nh = c_hoff[d] - c_hoff[d - 1];  // entries for this d (max order)
    int ncount = 1;
    // entries needed for order R: C(d+R, d); computed on the host into it.R-indexed table size
    {
        // graded order: count multi-indices with |alpha| <= R
        long long c = 1;
        for (int i = 1; i <= d; ++i) c = c * (it.R + i) / i;
        ncount = (int)c;
        if (ncount > nh) ncount = nh;
    }
    const HEnt* tab = c_htab + c_hoff[d - 1];
    for (int s = 0; s < it.nsig; ++s) {
        const double* L = it.lam[s];
        real z[MAXD];
        real q = 0;
#pragma unroll
        for (int a = 0; a < MAXD; ++a) {
            real acc = 0;
#pragma unroll
            for (int b = 0; b < MAXD; ++b)
                if (a < d && b < d) acc += (real)L[a * MAXD + b] * x[b];
            z[a] = acc;
            q += x[a] * acc;
        }
        ex[s] = (real)it.nrm[s] * exp(real(-0.5) * q);
        real* h = He[s];
        h[0] = real(1);
        for (int t = 1; t < ncount; ++t) {
            const HEnt e = tab[t];
            real v = z[e.piv] * h[e.par];
            for (int r = 0; r < e.nred; ++r) v -= real(e.rc[r]) * (real)L[e.piv * MAXD + e.rj[r]] * h[e.ridx[r]];
            h[t] = v;
        }
    }
    real a = 0, b = 0;
    for (int m = 0; m < it.nterm[0]; ++m) a += it.tw8[0][m] * He[it.tsig[0][m]][it.the[0][m]] * ex[it.tsig[0][m]];
    for (int m = 0; m < it.nterm[1]; ++m) b += it.tw8[1][m] * He[it.tsig[1][m]][it.the[1][m]] * ex[it.tsig[1][m]];
    va = a;
    vb = b;
}

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
__device__ __forceinline__ void df_acc(DFloat& a, float x) {
    const DFloat s = df_two_sum(a.h, x);
    const float e = s.l + a.l;
    a.h = s.h + e;
    a.l = e - (a.h - s.h);
}

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
__device__ __forceinline__ void block_reduce_acc(const SumAcc<double>& s, double* out2);

__device__ __forceinline__ int spec_weight_idx(int q, int wdiv) { return q / wdiv; }

// weight of a last-axis frequency in the half-spectrum sum: 1 for w = 0 and
// (P even) w = P/2, 2 otherwise
__device__ __forceinline__ int half_weight(int w, int P) { return (w == 0 || 2 * w == P) ? 1 : 2; }

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

// Spectral sink of a finished line batch: Y[c][w] for lines q = q0 + c.
// kind 0: accumulate sum spec[q][w] * weight * Y; kind 1: spec_out = |Y|^2.
template <typename real, typename C>
__device__ void spectral_sink(const Item<real>& it, const C* Y, int nl, int P, int q0, int wdiv, int Plast,
                              bool last_is_line, double* partial_out, const real* srow = nullptr) {
    if (it.kind == 0) {
        SumAcc<real> acc;
        for (int t = threadIdx.x; t < nl * P; t += blockDim.x) {
            const int c = t / P;
            const int w = t - c * P;
            const int q = q0 + c;
            // d = 1: the line index is the last axis itself (w is w_{d-1})
            const int wl = last_is_line ? w : q / wdiv;
            const real sv = srow ? srow[t] : it.spec[(long long)q * P + w];
            const real s = sv * real(half_weight(wl, Plast));
            const C y = Y[pad(t)];
            acc.add(s * y.x, s * y.y);
        }
        block_reduce_acc(acc, partial_out);
    } else {
        for (int t = threadIdx.x; t < nl * P; t += blockDim.x) {
            const int c = t / P;
            const int w = t - c * P;
            const C y = Y[pad(t)];
            it.spec_out[(long long)(q0 + c) * P + w] = y.x * y.x + y.y * y.y;
        }
    }
}

// ------------------------------------------------------------ stage A
template <typename real>
__global__ void __launch_bounds__(256) k_stage_a(const Item<real>* __restrict__ items, const Tile* __restrict__ tiles,
                                                 int ntiles, int cap, typename Cpx<real>::T* __restrict__ scratch,
                                                 const typename Cpx<real>::T* __restrict__ twpool,
                                                 double* __restrict__ partial) {
    using C = typename Cpx<real>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* bufa = reinterpret_cast<C*>(smem_raw);
    C* bufb = bufa + padded_cap(cap);
    C* tw = bufb + padded_cap(cap);
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile tl = tiles[ti];
        const Item<real>& it = items[tl.item];
        const int d = it.d;
        const int ax = d - 1;
        const AxisPlan& ap = it.ax[ax];
        const int P = ap.P;
        const int nl = tl.n;
        __syncthreads();
        load_twiddles(tw, twpool, ap);
        // fill lines
        for (int t = threadIdx.x; t < nl * P; t += blockDim.x) {
            const int c = t / P;
            const int p = t - c * P;
            int idx = p + it.off[ax];
            if (idx >= P) idx -= P;
            C v = C{real(0), real(0)};
            if (idx < it.S[ax]) {
                const int line = tl.a + c;
                if (it.kind == 1) {
                    const long long M_last = it.S[ax];
                    v.x = it.counts[(long long)line * M_last + idx];
                } else {
                    int j[MAXD];
                    int rem = line;
                    for (int k = d - 2; k >= 0; --k) {
                        const int ik = rem % it.S[k];
                        rem /= it.S[k];
                        j[k] = ik - it.off[k];
                    }
                    j[ax] = idx - it.off[ax];
                    real va, vb;
                    kernel_pair(it, j, va, vb);
                    v = C{va, vb};
                }
            }
            bufa[pad(t)] = v;
        }
        C* Y = smem_fft(bufa, bufb, nl, ap, tw);
        const int Q = P / 2 + 1;
        if (d == 1) {
            // the only axis: sink over w in [0, P/2]
            // compact the half spectrum in place is unnecessary: sink reads Y[w], w < Q
            if (it.kind == 0) {
                SumAcc<real> acc;
                for (int w = threadIdx.x; w < Q; w += blockDim.x) {
                    const real s = it.spec[w] * real(half_weight(w, P));
                    acc.add(s * Y[pad(w)].x, s * Y[pad(w)].y);
                }
                block_reduce_acc(acc, partial + 2 * (long long)it.tileF0);
            } else {
                for (int w = threadIdx.x; w < Q; w += blockDim.x) {
                    const C y = Y[pad(w)];
                    it.spec_out[w] = y.x * y.x + y.y * y.y;
                }
            }
        } else {
            // write [w][line] for w < Q
            long long nlines_tot = 1;
            for (int k = 0; k < d - 1; ++k) nlines_tot *= it.S[k];
            C* out = scratch + it.scr[0];
            for (int t = threadIdx.x; t < nl * Q; t += blockDim.x) {
                const int w = t / nl;
                const int c = t - w * nl;
                out[(long long)w * nlines_tot + tl.a + c] = Y[pad(c * P + w)];
            }
        }
    }
}

// ------------------------------------------------------------ mid pass (axis k, 0 < k < d-1)
template <typename real>
__global__ void __launch_bounds__(256) k_mid(const Item<real>* __restrict__ items, const Tile* __restrict__ tiles,
                                             int ntiles, int axis, int cap,
                                             typename Cpx<real>::T* __restrict__ scratch,
                                             const typename Cpx<real>::T* __restrict__ twpool) {
    using C = typename Cpx<real>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* bufa = reinterpret_cast<C*>(smem_raw);
    C* bufb = bufa + padded_cap(cap);
    C* tw = bufb + padded_cap(cap);
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile tl = tiles[ti];
        const Item<real>& it = items[tl.item];
        const int d = it.d;
        const AxisPlan& ap = it.ax[axis];
        const int P = ap.P;
        const int S = it.S[axis];
        const int nl = tl.n;
        // ping-pong: stage A wrote scr[0]; the pass for axis d-2 reads 0 writes 1, etc.
        const int rsel = ((d - 2 - axis) & 1);
        const C* in = scratch + it.scr[rsel];
        C* out = scratch + it.scr[rsel ^ 1];
        long long O = 1;
        for (int k = 0; k < axis; ++k) O *= it.S[k];
        __syncthreads();
        load_twiddles(tw, twpool, ap);
        const long long ibase = ((long long)tl.a * O + tl.b) * S;
        for (int t = threadIdx.x; t < nl * S; t += blockDim.x) cp_async<sizeof(C)>(bufb + t, in + ibase + t);
        cp_async_wait_all();
        __syncthreads();
        for (int t = threadIdx.x; t < nl * P; t += blockDim.x) {
            const int c = t / P;
            const int p = t - c * P;
            int idx = p + it.off[axis];
            if (idx >= P) idx -= P;
            bufa[pad(t)] = (idx < S) ? bufb[c * S + idx] : C{real(0), real(0)};
        }
        C* Y = smem_fft(bufa, bufb, nl, ap, tw);
        const long long obase = (long long)tl.a * P;
        for (int t = threadIdx.x; t < nl * P; t += blockDim.x) {
            const int w = t / nl;
            const int c = t - w * nl;
            out[(obase + w) * O + tl.b + c] = Y[pad(c * P + w)];
        }
    }
}

// ------------------------------------------------------------ final pass (axis 0) + sink
template <typename real>
__global__ void __launch_bounds__(256) k_final(const Item<real>* __restrict__ items, const Tile* __restrict__ tiles,
                                               int ntiles, int cap, typename Cpx<real>::T* __restrict__ scratch,
                                               const typename Cpx<real>::T* __restrict__ twpool,
                                               double* __restrict__ partial) {
    using C = typename Cpx<real>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* bufa = reinterpret_cast<C*>(smem_raw);
    C* bufb = bufa + padded_cap(cap);
    C* tw = bufb + padded_cap(cap);
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile tl = tiles[ti];
        const Item<real>& it = items[tl.item];
        const int d = it.d;
        const AxisPlan& ap = it.ax[0];
        const int P = ap.P;
        const int S = it.S[0];
        const int nl = tl.n;
        // input buffer: written by the last mid pass (axis 1) or by stage A (d = 2)
        const int rsel = (d - 2) & 1;
        const C* in = scratch + it.scr[rsel];
        __syncthreads();
        // stage this tile's input block (nl x S, contiguous) in bufb and, for a
        // kernel item, its spectrum rows (nl x P reals) behind the twiddles
        const C* ib = in + (long long)tl.a * S;
        for (int t = threadIdx.x; t < nl * S; t += blockDim.x) cp_async<sizeof(C)>(bufb + t, ib + t);
        real* srow = reinterpret_cast<real*>(tw + P);
        if (it.kind == 0) {
            const real* sb = it.spec + (long long)tl.a * P;
            for (int t = threadIdx.x; t < nl * P; t += blockDim.x) cp_async<sizeof(real)>(srow + t, sb + t);
        }
        load_twiddles(tw, twpool, ap);
        cp_async_wait_all();
        __syncthreads();
        for (int t = threadIdx.x; t < nl * P; t += blockDim.x) {
            const int c = t / P;
            const int p = t - c * P;
            int idx = p + it.off[0];
            if (idx >= P) idx -= P;
            bufa[pad(t)] = (idx < S) ? bufb[c * S + idx] : C{real(0), real(0)};
        }
        C* Y = smem_fft(bufa, bufb, nl, ap, tw);
        int wdiv = 1;
        for (int k = 1; k < d - 1; ++k) wdiv *= it.ax[k].P;
        spectral_sink<real, C>(it, Y, nl, P, tl.a, wdiv, it.ax[d - 1].P, false,
                               partial + 2 * (long long)ti, it.kind == 0 ? srow : nullptr);
    }
}

// ------------------------------------------------------------ reduce
template <typename real>
__global__ void k_reduce(const Item<real>* __restrict__ items, int nitems, const double* __restrict__ partial,
                         double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nitems) return;
    const Item<real>& it = items[i];
    if (it.kind != 0) return;
    double a = 0.0, b = 0.0;
    for (int t = 0; t < it.ntileF; ++t) {
        a += partial[2 * (long long)(it.tileF0 + t)];
        b += partial[2 * (long long)(it.tileF0 + t) + 1];
    }
    out[2 * i] = a * it.scale;
    out[2 * i + 1] = b * it.scale;
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

// value of the packed pair at lag (j0, j1), d = 2, orders <= R
template <typename real, int R>
__device__ __forceinline__ void kernel_pair_2d(const FusedItem<real>& f, int j0, int j1, real& va, real& vb) {
    constexpr HTab<2, R> ht{};
    constexpr int N = HTab<2, R>::N;
    // the quadratic form in the working type (FP64 is slow on this part; its
    // FP32 rounding, about q u / 2 relative, only touches the kernel's tails)
    const real x0 = (real)f.delta0 * (real)j0, x1 = (real)f.delta1 * (real)j1;
    real a = 0, b = 0;
#pragma unroll
    for (int s = 0; s < MAXSIG; ++s) {
        if (s < f.nsig) {
            real z0, z1, e;
            if constexpr (sizeof(real) == 8) {
                z0 = f.lam[s][0] * x0 + f.lam[s][1] * x1;
                z1 = f.lam[s][2] * x0 + f.lam[s][3] * x1;
                e = f.nrm[s] * exp(real(-0.5) * (x0 * z0 + x1 * z1));
            } else {
                z0 = f.laml[s][0] * x0 + f.laml[s][1] * x1;
                z1 = f.laml[s][2] * x0 + f.laml[s][3] * x1;
                e = f.nrm[s] * expf(-0.5f * (x0 * z0 + x1 * z1));
            }
            real He[N];
            He[0] = real(1);
#pragma unroll
            for (int t = 1; t < N; ++t) {
                real v = (ht.piv[t] == 0 ? z0 : z1) * He[ht.par[t]];
#pragma unroll
                for (int r = 0; r < 2; ++r)
                    if (r < ht.nred[t]) v -= real(ht.rc[t][r]) * f.laml[s][ht.piv[t] * 2 + ht.rj[t][r]] * He[ht.ridx[t][r]];
                He[t] = v;
            }
            real pa = 0, pb = 0;
#pragma unroll
            for (int t = 0; t < N; ++t) {
                pa += f.W[0][s][t] * He[t];
                pb += f.W[1][s][t] * He[t];
            }
            a += e * pa;
            b += e * pb;
        }
    }
    va = a;
    vb = b;
}

// ------------------------------------------------------------ fused 2-D path (one cluster per item)
// d = 2 only.  The cs CTAs of a cluster split the S_0 generated lines of the
// axis-1 pass (k_stage_a's work).  Each CTA pushes the half spectrum of its
// lines (w_1 <= P_1/2) straight into the gather buffer of the CTA that owns
// each w_1 column (distributed shared memory stores); after one cluster
// barrier every CTA holds the S_0 inputs of its axis-0 lines locally,
// transforms them and reduces against the count spectrum (k_final's work),
// whose rows were staged into shared memory by one bulk (TMA) copy issued
// at kernel start.  The per-CTA partial sums meet in rank 0's shared memory
// and rank 0 writes the item's two scaled sums (k_reduce's work).
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// bounded wait on an mbarrier phase; returns false when the limit is hit
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <typename real, int R>
__global__ void __launch_bounds__(256) k_fused2d(const FusedItem<real>* __restrict__ items, int cs, int gat_elems,
                                                 int spc_elems, int cap, int pmax,
                                                 const typename Cpx<real>::T* __restrict__ twpool,
                                                 double* __restrict__ out, int* __restrict__ errflag) {
    using C = typename Cpx<real>::T;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double cl_red[16][2];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ FusedItem<real> f;
    C* gat = reinterpret_cast<C*>(smem_raw);                 // [S_0][cpc] inputs of my axis-0 lines
    real* spc = reinterpret_cast<real*>(gat + gat_elems);    // [cpc][P_0] my spectrum rows
    C* tw1 = reinterpret_cast<C*>(spc + spc_elems);
    C* tw0 = tw1 + pmax;
    C* bufa = tw0 + pmax;
    C* bufb = bufa + padded_cap(cap);
    const int rank = (int)cluster.block_rank();
    const int item = blockIdx.x / cs;
    {
        // stage the item (prepared on the host) in shared memory, 4 bytes per thread
        const uint32_t* src = reinterpret_cast<const uint32_t*>(items + item);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&f);
        for (int t = threadIdx.x; t < (int)(sizeof(FusedItem<real>) / 4); t += blockDim.x) dst[t] = src[t];
        __syncthreads();
    }
    const int P1 = f.a1.P, P0 = f.a0.P, Q1 = P1 / 2 + 1;
    const int S0 = f.S0, S1 = f.S1;
    const int lpc = (S0 + cs - 1) / cs;
    const int cpc = (Q1 + cs - 1) / cs;
    const int q0 = rank * cpc;
    const int nq = max(0, min(Q1, q0 + cpc) - q0);
    // ---- stage my spectrum rows [q0, q0 + nq) x P_0 into shared memory
    const size_t sbytes = sizeof(real) * (size_t)nq * P0;
    const real* sg = f.spec + (size_t)q0 * P0;
    const bool bulk = nq > 0 && (sbytes % 16 == 0) && (((uintptr_t)sg) % 16 == 0);
    const uint32_t bar = smem_u32(&mbar);
    if (bulk && threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)sbytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(spc)),
            "l"(sg), "r"((uint32_t)sbytes), "r"(bar)
            : "memory");
    } else if (!bulk) {
        for (int t = threadIdx.x; t < nq * P0; t += blockDim.x) spc[t] = sg[t];
    }
    load_twiddles(tw1, twpool, f.a1);
    load_twiddles(tw0, twpool, f.a0);
    // ---- axis-1 pass over my generated lines
    const int l0 = rank * lpc;
    const int nl = max(0, min(S0, l0 + lpc) - l0);
    const uint32_t mP1 = magic_of((uint32_t)P1), mQ1 = magic_of((uint32_t)Q1);
    const uint32_t mcpc = magic_of((uint32_t)max(cpc, 2));
    const int off0 = f.off0, off1 = f.off1;
    if (nl > 0) {
        for (int t = threadIdx.x; t < nl * P1; t += blockDim.x) {
            const int c = (int)qdiv((uint32_t)t, mP1);
            const int p = t - c * P1;
            int idx = p + off1;
            if (idx >= P1) idx -= P1;
            C v = C{real(0), real(0)};
            if (idx < S1) {
                real va, vb;
                kernel_pair_2d<real, R>(f, l0 + c - off0, idx - off1, va, vb);
                v = C{va, vb};
            }
            bufa[pad(t)] = v;
        }
        C* Y = smem_fft(bufa, bufb, nl, f.a1, tw1);
        // push (line, w_1) to the owner of column w_1: gat[line][w_1 - q0_owner]
        for (int t = threadIdx.x; t < nl * Q1; t += blockDim.x) {
            const int c = (int)qdiv((uint32_t)t, mQ1);
            const int q = t - c * Q1;
            const int dst = (cpc == 1) ? q : (int)qdiv((uint32_t)q, mcpc);
            C* g = cluster.map_shared_rank(gat, dst);
            g[(l0 + c) * cpc + (q - dst * cpc)] = Y[pad(c * P1 + q)];
        }
    }
    cluster.sync();
    // ---- axis-0 pass over my columns
    SumAcc<real> acc;
    const uint32_t mP0 = magic_of((uint32_t)P0);
    if (nq > 0) {
        for (int t = threadIdx.x; t < nq * P0; t += blockDim.x) {
            const int c = (int)qdiv((uint32_t)t, mP0);
            const int p = t - c * P0;
            int idx = p + off0;
            if (idx >= P0) idx -= P0;
            bufa[pad(t)] = (idx < S0) ? gat[idx * cpc + c] : C{real(0), real(0)};
        }
        C* Y = smem_fft(bufa, bufb, nq, f.a0, tw0);
        if (bulk && !mbar_wait(bar, 0)) {
            if (threadIdx.x == 0) atomicOr(errflag, 1);
        } else {
            for (int t = threadIdx.x; t < nq * P0; t += blockDim.x) {
                const int c = (int)qdiv((uint32_t)t, mP0);
                const int q = q0 + c;
                const real s = spc[t] * real(half_weight(q, P1));
                const C y = Y[pad(t)];
                acc.add(s * y.x, s * y.y);
            }
        }
    }
    double part[2];
    block_reduce_acc(acc, part);
    if (threadIdx.x == 0) {
        double* dst = cluster.map_shared_rank(&cl_red[0][0], 0);
        dst[2 * rank] = part[0];
        dst[2 * rank + 1] = part[1];
    }
    cluster.sync();
    if (rank == 0 && threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int r = 0; r < cs; ++r) {
            a += cl_red[r][0];
            b += cl_red[r][1];
        }
        out[2 * item] = a * f.scale;
        out[2 * item + 1] = b * f.scale;
    }
}

// ------------------------------------------------------------ launchers
template <typename real>
static size_t smem_bytes(int cap, int pmax) {
    return sizeof(typename Cpx<real>::T) * (size_t)(2 * padded_cap(cap) + pmax);
}

template <typename real>
cudaError_t launch_stage_a(const Item<real>* items, const Tile* tiles, int ntiles, int pmax, int cap,
                           typename Cpx<real>::T* scratch, const typename Cpx<real>::T* twpool, double* partial,
                           int grid, cudaStream_t st) {
    const size_t sm = smem_bytes<real>(cap, pmax);
    cudaError_t e = cudaFuncSetAttribute(k_stage_a<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_stage_a<real><<<grid, 256, sm, st>>>(items, tiles, ntiles, cap, scratch, twpool, partial);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_mid(const Item<real>* items, const Tile* tiles, int ntiles, int axis, int pmax, int cap,
                       typename Cpx<real>::T* scratch, const typename Cpx<real>::T* twpool, int grid,
                       cudaStream_t st) {
    const size_t sm = smem_bytes<real>(cap, pmax);
    cudaError_t e = cudaFuncSetAttribute(k_mid<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_mid<real><<<grid, 256, sm, st>>>(items, tiles, ntiles, axis, cap, scratch, twpool);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_final(const Item<real>* items, const Tile* tiles, int ntiles, int pmax, int cap,
                         typename Cpx<real>::T* scratch, const typename Cpx<real>::T* twpool, double* partial,
                         int grid, cudaStream_t st) {
    // ping-pong buffers, twiddles, then the staged spectrum rows (cap reals)
    const size_t sm = smem_bytes<real>(cap, pmax) + sizeof(real) * (size_t)cap;
    cudaError_t e = cudaFuncSetAttribute(k_final<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_final<real><<<grid, 256, sm, st>>>(items, tiles, ntiles, cap, scratch, twpool, partial);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_reduce(const Item<real>* items, int nitems, const double* partial, double* out, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    k_reduce<real><<<(nitems + 127) / 128, 128, 0, st>>>(items, nitems, partial, out);
    return cudaGetLastError();
}


template <typename real, int R>
static cudaError_t launch_fused2d_r(const FusedItem<real>* items, int nitems, int cs, int gat_elems, int spc_elems,
                                   int cap, int pmax, const typename Cpx<real>::T* twpool, double* out, int* errflag,
                                   cudaStream_t st) {
    using C = typename Cpx<real>::T;
    // spectrum rows are real; keep the complex buffers after them 16-byte aligned
    const int spc_pad = (spc_elems + 3) & ~3;
    const size_t sm = sizeof(C) * (size_t)(gat_elems + 2 * pmax + 2 * padded_cap(cap)) + sizeof(real) * (size_t)spc_pad;
    static size_t set_bytes = 0;
    if (sm > set_bytes) {
        cudaError_t e = cudaFuncSetAttribute(k_fused2d<real, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_fused2d<real, R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        set_bytes = sm;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nitems * cs), 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cs > 8) {
        // clusters above the portable size must be schedulable with this shared-memory footprint
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_fused2d<real, R>, &cfg) != cudaSuccess || nclusters < 1) {
            cudaGetLastError();
            return cudaErrorNotSupported;
        }
    }
    return cudaLaunchKernelEx(&cfg, k_fused2d<real, R>, items, cs, gat_elems, spc_pad, cap, pmax, twpool, out,
                              errflag);
}

template <typename real>
cudaError_t launch_fused2d(const FusedItem<real>* items, int nitems, int rmax, int cs, int gat_elems, int spc_elems,
                           int cap, int pmax, const typename Cpx<real>::T* twpool, double* out, int* errflag,
                           cudaStream_t st) {
    if (rmax <= 2)
        return launch_fused2d_r<real, 2>(items, nitems, cs, gat_elems, spc_elems, cap, pmax, twpool, out, errflag, st);
    if (rmax <= 4 && sizeof(real) == 4)
        return launch_fused2d_r<real, 4>(items, nitems, cs, gat_elems, spc_elems, cap, pmax, twpool, out, errflag, st);
    return cudaErrorNotSupported;
}

#define KDEFFT_INST(real)                                                                                       \
    template cudaError_t launch_stage_a<real>(const Item<real>*, const Tile*, int, int, int,                   \
                                              typename Cpx<real>::T*, const typename Cpx<real>::T*, double*, \
                                              int, cudaStream_t);                                             \
    template cudaError_t launch_mid<real>(const Item<real>*, const Tile*, int, int, int, int,                  \
                                          typename Cpx<real>::T*, const typename Cpx<real>::T*, int,           \
                                          cudaStream_t);                                                      \
    template cudaError_t launch_final<real>(const Item<real>*, const Tile*, int, int, int,                     \
                                            typename Cpx<real>::T*, const typename Cpx<real>::T*, double*,     \
                                            int, cudaStream_t);                                               \
    template cudaError_t launch_reduce<real>(const Item<real>*, int, const double*, double*, cudaStream_t);        \
    template cudaError_t launch_fused2d<real>(const FusedItem<real>*, int, int, int, int, int, int, int,           \
                                              const typename Cpx<real>::T*, double*, int*, cudaStream_t);

KDEFFT_INST(float)
KDEFFT_INST(double)

}  // namespace kdefft
