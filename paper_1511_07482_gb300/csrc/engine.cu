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
#include <algorithm>

#include <cooperative_groups.h>
#include <type_traits>
#include <map>
#include <mutex>
#include <tuple>

#include "engine.cuh"
#include "devutil.cuh"

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

// the same twiddles as FP32 pairs, split at compile time (no FP64
// conversion at run time when the table is indexed)
template <int R>
struct CxTwPair {
    float ch[R], cl[R], sh[R], sl[R];
    constexpr CxTwPair() : ch(), cl(), sh(), sl() {
        for (int m = 0; m < R; ++m) {
            const CxCis z = cx_cis(m, R);
            ch[m] = (float)z.c;
            cl[m] = (float)(z.c - (double)(float)z.c);
            sh[m] = (float)z.s;
            sl[m] = (float)(z.s - (double)(float)z.s);
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
        constexpr CxTwPair<R> tp{};
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
                    R_ cw, sw;
                    if constexpr (sizeof(R_) == 8 && !std::is_same<R_, double>::value) {   // FP32 pairs
                        cw = R_(tp.ch[m], tp.cl[m]);
                        sw = R_(tp.sh[m], tp.sl[m]);
                    } else {
                        cw = R_(tw.c[m]);
                        sw = R_(tw.s[m]);
                    }
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


__device__ __forceinline__ int spec_weight_idx(int q, int wdiv) { return q / wdiv; }

// weight of a last-axis frequency in the half-spectrum sum: 1 for w = 0 and
// (P even) w = P/2, 2 otherwise
__device__ __forceinline__ int half_weight(int w, int P) { return (w == 0 || 2 * w == P) ? 1 : 2; }


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

// ------------------------------------------------------------ autocorrelation passes
// One pass of the count autocorrelation a = F^-1(|C|^2) (FP64) along one
// axis, for many datasets in one launch.  A line holds the W spectrum values
// along the axis (weights h_w: 2 on the interior of a half-spectrum axis,
// else 1), zero-extended to the padded size P; its inverse DFT of length P
// runs in shared memory and the J lags jlo .. jlo + J - 1 are kept.  The
// inverse comes from the forward transform:
//   sum_w x_w e^{+2 pi i w j / P} = conj(sum_w conj(x_w) e^{-2 pi i w j / P}).
// Line l = o I + i of a pass reads (o, w, i) at (o W + w) I + i and writes
// lag jj to (o J + jj) I + i; the real spectrum of the first pass has I = 1.
template <typename J>
__device__ __forceinline__ int job_of(const J* __restrict__ jobs, int n, long long b) {
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

// C: double2 (FP64) or dcplx (FP32 pairs, the same layout and size)
template <typename C>
__global__ void __launch_bounds__(256) k_acorr_fft(const AcorrJob* __restrict__ jobs, int njobs,
                                                   const C* __restrict__ twpool) {
    using R = decltype(C{}.x);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const AcorrJob& jb = jobs[job_of(jobs, njobs, blockIdx.x)];
    const int P = jb.ap.P, W = jb.W, J = jb.J, cap = jb.nl;
    const long long I = jb.I;
    const R* in_r = reinterpret_cast<const R*>(jb.in_r);
    const C* in_c = reinterpret_cast<const C*>(jb.in_c);
    C* out_c = reinterpret_cast<C*>(jb.out_c);
    C* bufa = reinterpret_cast<C*>(smem_raw);
    C* bufb = bufa + padded_cap(cap * P);
    C* tw = bufb + padded_cap(cap * P);
    const long long l0 = ((long long)blockIdx.x - jb.blk0) * cap;
    const int nl = (int)min((long long)cap, jb.O * I - l0);
    load_twiddles(tw, twpool, jb.ap);
    auto hw = [&](int w) { return (jb.half && w != 0 && 2 * w != P) ? R(2.0) : R(1.0); };
    if (I == 1) {   // consecutive lines are rows: w fastest
        for (int t = threadIdx.x; t < nl * P; t += blockDim.x) {
            const int c = t / P, w = t - c * P;
            C x{R(0.0), R(0.0)};
            if (w < W) {
                const long long at = (l0 + c) * W + w;
                const R h = hw(w);
                x = in_r ? C{h * in_r[at], R(0.0)} : C{h * in_c[at].x, -(h * in_c[at].y)};
            }
            bufa[pad(t)] = x;
        }
    } else {        // consecutive lines are consecutive i: line fastest
        for (int t = threadIdx.x; t < nl * P; t += blockDim.x) {
            const int w = t / nl, c = t - w * nl;
            C x{R(0.0), R(0.0)};
            if (w < W) {
                const long long l = l0 + c, o = l / I, i = l - o * I;
                const C v = in_c[(o * W + w) * I + i];
                const R h = hw(w);
                x = C{h * v.x, -(h * v.y)};
            }
            bufa[pad(c * P + w)] = x;
        }
    }
    const C* Y = smem_fft(bufa, bufb, nl, jb.ap, tw);
    for (int t = threadIdx.x; t < nl * J; t += blockDim.x) {
        int c, jj;
        if (I == 1) {
            c = t / J;
            jj = t - c * J;
        } else {
            jj = t / nl;
            c = t - jj * nl;
        }
        int j = (jb.jlo + jj) % P;
        if (j < 0) j += P;
        const C y = Y[pad(c * P + j)];
        const long long l = l0 + c, o = l / I, i = l - o * I;
        const long long at = (o * J + jj) * I + i;
        if (jb.out_r) {
            const double v = to_double(y.x) * jb.scale;
            jb.out_r[at] = v;
            if (jb.out_r32) jb.out_r32[at] = (float)v;
        } else {
            out_c[at] = C{y.x, -y.y};
        }
    }
}

// Forward passes of the count spectrum in FP32 pairs (SpecJob).
__global__ void __launch_bounds__(256) k_spec_df(const SpecJob* __restrict__ jobs, int njobs,
                                                 const dcplx* __restrict__ twpool) {
    using C = dcplx;
    using R = dflt;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SpecJob& jb = jobs[job_of(jobs, njobs, blockIdx.x)];
    const int P = jb.ap.P, X = jb.X, Yn = jb.Y, cap = jb.nl;
    const long long I = jb.I;
    const C* in_c = reinterpret_cast<const C*>(jb.in_c);
    C* bufa = reinterpret_cast<C*>(smem_raw);
    C* bufb = bufa + padded_cap(cap * P);
    C* tw = bufb + padded_cap(cap * P);
    const long long l0 = ((long long)blockIdx.x - jb.blk0) * cap;
    const int nl = (int)min((long long)cap, jb.O * I - l0);
    load_twiddles(tw, twpool, jb.ap);
    if (I == 1) {   // rows: x fastest
        for (int t = threadIdx.x; t < nl * P; t += blockDim.x) {
            const int c = t / P, x = t - c * P;
            C v{R(0.0), R(0.0)};
            if (x < X) {
                const long long at = (l0 + c) * X + x;
                v = jb.in_f ? C{R(jb.in_f[at], 0.f), R(0.0)} : in_c[at];
            }
            bufa[pad(t)] = v;
        }
    } else {        // line fastest
        for (int t = threadIdx.x; t < nl * P; t += blockDim.x) {
            const int x = t / nl, c = t - x * nl;
            C v{R(0.0), R(0.0)};
            if (x < X) {
                const long long l = l0 + c, o = l / I, i = l - o * I;
                const long long at = (o * X + x) * I + i;
                v = jb.in_f ? C{R(jb.in_f[at], 0.f), R(0.0)} : in_c[at];
            }
            bufa[pad(c * P + x)] = v;
        }
    }
    const C* Yb = smem_fft(bufa, bufb, nl, jb.ap, tw);
    C* out_c = reinterpret_cast<C*>(jb.out_c);
    R* out_s = reinterpret_cast<R*>(jb.out_s);
    for (int t = threadIdx.x; t < nl * Yn; t += blockDim.x) {
        int c, y;
        if (I == 1) {
            c = t / Yn;
            y = t - c * Yn;
        } else {
            y = t / nl;
            c = t - y * nl;
        }
        const C v = Yb[pad(c * P + y)];
        const long long l = l0 + c, o = l / I, i = l - o * I;
        if (out_c) {
            out_c[(o * Yn + y) * I + i] = v;
        } else {
            // |X|^2 at the inner index reordered with w_{d-1} slowest
            long long r = i, q = 0;
            int wv[MAXD];
            for (int m = jb.d - 1; m >= 1; --m) {
                wv[m] = (int)(r % jb.ext[m]);
                r /= jb.ext[m];
            }
            for (int m = jb.d - 1; m >= 1; --m) q = q * jb.ext[m] + wv[m];
            out_s[q * P + y] = v.x * v.x + v.y * v.y;
        }
    }
}

cudaError_t acorr_plan(AcorrJob* jobs_h, int n, long long* blocks_out, size_t* sm_out) {
    long long blocks = 0;
    size_t sm = 0;
    for (int k = 0; k < n; ++k) {
        AcorrJob& jb = jobs_h[k];
        if (jb.nl < 1 || jb.ap.P < 2 || jb.W > jb.ap.P || (!jb.in_r && !jb.in_c) || (jb.in_r && jb.I != 1))
            return cudaErrorInvalidValue;
        jb.blk0 = blocks;
        blocks += (jb.O * jb.I + jb.nl - 1) / jb.nl;
        sm = std::max(sm, acorr_smem_bytes(jb.ap.P, jb.nl));
    }
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    *blocks_out = blocks;
    *sm_out = sm;
    return cudaSuccess;
}

cudaError_t spec_plan(SpecJob* jobs_h, int n, long long* blocks_out, size_t* sm_out) {
    long long blocks = 0;
    size_t sm = 0;
    for (int k = 0; k < n; ++k) {
        SpecJob& jb = jobs_h[k];
        if (jb.nl < 1 || jb.ap.P < 2 || jb.X > jb.ap.P || jb.Y > jb.ap.P || (!jb.in_f && !jb.in_c) ||
            (!jb.out_c && !jb.out_s) || (jb.out_s && jb.O != 1) || jb.d < 1 || jb.d > MAXD)
            return cudaErrorInvalidValue;
        jb.blk0 = blocks;
        blocks += (jb.O * jb.I + jb.nl - 1) / jb.nl;
        sm = std::max(sm, acorr_smem_bytes(jb.ap.P, jb.nl));
    }
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    *blocks_out = blocks;
    *sm_out = sm;
    return cudaSuccess;
}

cudaError_t launch_acorr(const AcorrJob* jobs_d, int n, long long blocks, size_t sm, const double2* twpool,
                         cudaStream_t st) {
    if (n <= 0 || blocks <= 0) return cudaSuccess;
    k_acorr_fft<double2><<<(unsigned)blocks, 256, sm, st>>>(jobs_d, n, twpool);
    return cudaGetLastError();
}

cudaError_t launch_acorr_df(const AcorrJob* jobs_d, int n, long long blocks, size_t sm, const void* twpool,
                            cudaStream_t st) {
    if (n <= 0 || blocks <= 0) return cudaSuccess;
    k_acorr_fft<dcplx><<<(unsigned)blocks, 256, sm, st>>>(jobs_d, n, (const dcplx*)twpool);
    return cudaGetLastError();
}

cudaError_t launch_spec_df(const SpecJob* jobs_d, int n, long long blocks, size_t sm, const void* twpool,
                           cudaStream_t st) {
    if (n <= 0 || blocks <= 0) return cudaSuccess;
    k_spec_df<<<(unsigned)blocks, 256, sm, st>>>(jobs_d, n, (const dcplx*)twpool);
    return cudaGetLastError();
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

// ------------------------------------------------------------ device-resident selection (d = 2, FP32)
// One cluster per start.  Each round, rank 0 (one thread, FP64 host-style
// algebra) turns the trial Cholesky parameters into H, checks the search
// domain, picks L (Eq. 26) and P, and writes the two packed work items of the
// objective and its gradient (value + dH_00, dH_01 + dH_11); the cluster
// evaluates both with the fused pipeline below; rank 0 assembles the value
// and gradient and applies the line search / BFGS update that the host
// optimiser uses.  Every loop is bounded.

// The four grids of the search at lag x = (delta_0 j_0, delta_1 j_1): the
// objective's kernel and its derivatives in H_00, H_01 (tied), H_11, from
// the Gaussians of the covariances Sigma_s (LSCV: 2H, H; SCV: 2H + 2G,
// H + 2G, 2G) and the order-2 Hermite terms He_(2,0) = z_0^2 - L_00,
// He_(1,1) = z_0 z_1 - L_01, He_(0,2) = z_1^2 - L_11, z = L x (heat
// equation: d phi_S / dS_ab = 1/2 d_a d_b phi_S).  For LSCV, Sigma_1 =
// Sigma_0 / 2, so L_1 = 2 L_0, z_1 = 2 z_0 and phi_H's exponent is twice
// phi_2H's: one exponential serves both.
//
// The SCV kernel phi_{2H+2G} - 2 phi_{H+2G} + phi_{2G} integrates to zero
// and is far smaller than its terms (the pilot smooths all three alike), so
// rounding each Gaussian on its own would leave errors of the terms' size.
// It is evaluated as phi_{2G} (m_0 - 2 m_1), where
//   m_s = phi_{Sigma_s} / phi_{2G} - 1 = rho_s expm1(-q_s / 2) + (rho_s - 1)
// and q_s = j^T D_s j is the exponent difference in lag-index coordinates:
// the products of j are exact, and D_s, rho_s and rho_s - 1 carry FP32
// remainders (sel_prepare), so the per-bandwidth constants add no
// systematic error, and m_0, 2 m_1 share only their first-order parts.  The
// gradient grids are formed in the same coordinates (Hermite terms
// Z_a Z_b - L~_ab with Z = L~ j, L~ = Delta Sigma^-1 Delta), which is
// delta_a delta_b times their value; the assembly divides it out.
template <int METHOD>
__device__ __forceinline__ void sel_grids(const FusedItem<float>& f, int j0i, int j1i, float d0, float d1, float* v) {
    if constexpr (METHOD == 0) {
        const float x0 = d0 * (float)j0i, x1 = d1 * (float)j1i;
        const float a00 = f.laml[0][0], a01 = f.laml[0][1], a11 = f.laml[0][3];
        const float z0 = fmaf(a00, x0, a01 * x1), z1 = fmaf(a01, x0, a11 * x1);
        const float q0 = fmaf(x0, z0, x1 * z1);
        const float u = expf(-0.5f * q0);
        const float e0 = f.nrm[0] * u;
        const float h3 = fmaf(z0, z0, -a00), h4 = fmaf(z0, z1, -a01), h5 = fmaf(z1, z1, -a11);
        const float e1 = f.nrm[1] * (u * u);
        const float g3 = fmaf(4.f * z0, z0, -2.f * a00), g4 = fmaf(4.f * z0, z1, -2.f * a01),
                    g5 = fmaf(4.f * z1, z1, -2.f * a11);
        v[0] = fmaf(-2.f, e1, e0);
        v[1] = fmaf(e0, h3, -e1 * g3);
        v[2] = 2.f * fmaf(e0, h4, -e1 * g4);
        v[3] = fmaf(e0, h5, -e1 * g5);
    } else {
        const float j0 = (float)j0i, j1 = (float)j1i;
        const float c00 = f.laml[2][0], c01 = f.laml[2][1], c11 = f.laml[2][3];
        const float w0 = fmaf(c00, j0, c01 * j1), w1 = fmaf(c01, j0, c11 * j1);
        const float e2 = f.nrm[2] * expf(-0.5f * fmaf(j0, w0, j1 * w1));
        float m[2], Z[2][2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float* D = f.xd[q];
            const float p0 = fmaf(D[0], j0, D[1] * j1), p1 = fmaf(D[1], j0, D[2] * j1);
            const float r0 = fmaf(D[3], j0, D[4] * j1), r1 = fmaf(D[4], j0, D[5] * j1);
            const float qh = fmaf(j0, p0, j1 * p1), ql = fmaf(j0, r0, j1 * r1);
            const float em = expm1f(-0.5f * qh);
            const float em2 = fmaf(-0.5f * ql, 1.f + em, em);   // expm1(-(qh + ql) / 2)
            m[q] = fmaf(D[6], em2, D[8]) + fmaf(D[7], em2, D[9]);
            Z[q][0] = w0 + p0;
            Z[q][1] = w1 + p1;
        }
        v[0] = e2 * fmaf(-2.f, m[1], m[0]);
        const float e0 = fmaf(e2, m[0], e2), e1 = fmaf(e2, m[1], e2);
        const float a00 = f.laml[0][0], a01 = f.laml[0][1], a11 = f.laml[0][3];
        const float b00 = f.laml[1][0], b01 = f.laml[1][1], b11 = f.laml[1][3];
        v[1] = fmaf(e0, fmaf(Z[0][0], Z[0][0], -a00), -e1 * fmaf(Z[1][0], Z[1][0], -b00));
        v[2] = 2.f * fmaf(e0, fmaf(Z[0][0], Z[0][1], -a01), -e1 * fmaf(Z[1][0], Z[1][1], -b01));
        v[3] = fmaf(e0, fmaf(Z[0][1], Z[0][1], -a11), -e1 * fmaf(Z[1][1], Z[1][1], -b11));
    }
}

// The four grids of one bandwidth (sel_grids: value and the three
// derivative grids, packed as two complex pairs) evaluated together by the
// cluster: lines and columns of the two pairs share every barrier, the
// twiddles, the staged spectrum rows and the reduction.  gat holds
// 2 x S_0 x cpc values (pair-major).  res4 (rank 0): the four scaled sums
// (pair 0 grids A, B; pair 1 grids A, B).
template <int METHOD>
__device__ __forceinline__ void sel_eval2(cg::cluster_group& cluster, const FusedItem<float>& f, int cs, int rank,
                                          int chunk, float2* gat,
                                          float* spc, float2* tw1, float2* tw0, float2* bufa, float2* bufb,
                                          const float2* twpool, double* cl_red, double* res4) {
    using C = float2;
    const int P1 = f.a1.P, P0 = f.a0.P, Q1 = P1 / 2 + 1;
    const int S0 = f.S0, S1 = f.S1;
    const int lpc = (S0 + cs - 1) / cs;
    const int cpc = (Q1 + cs - 1) / cs;
    const int q0 = rank * cpc;
    const int nq = max(0, min(Q1, q0 + cpc) - q0);
    const int l0 = rank * lpc;
    const int nl = max(0, min(S0, l0 + lpc) - l0);
    const int gpair = S0 * cpc;   // gather elements per pair
    const float* sg = f.spec + (size_t)q0 * P0;
    for (int t = threadIdx.x; t < nq * P0; t += blockDim.x) cp_async<4>(spc + t, sg + t);
    load_twiddles(tw1, twpool, f.a1);
    load_twiddles(tw0, twpool, f.a0);
    __syncthreads();
    const uint32_t mP1 = magic_of((uint32_t)P1), mQ1 = magic_of((uint32_t)Q1), mP0 = magic_of((uint32_t)P0);
    const uint32_t mcpc = magic_of((uint32_t)max(cpc, 2));
    const int off0 = f.off0, off1 = f.off1;
    // axis-1 pass: lines [pair 0: nc lines][pair 1: nc lines]
    for (int c0 = 0; c0 < nl; c0 += chunk) {
        const int nc = min(chunk, nl - c0);
        for (int t = threadIdx.x; t < nc * P1; t += blockDim.x) {
            const int c = (int)qdiv((uint32_t)t, mP1);
            const int p = t - c * P1;
            int idx = p + off1;
            if (idx >= P1) idx -= P1;
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            if (idx < S1) sel_grids<METHOD>(f, l0 + c0 + c - off0, idx - off1, (float)f.delta0, (float)f.delta1, v);
            bufa[pad(t)] = C{v[0], v[1]};
            bufa[pad(t + nc * P1)] = C{v[2], v[3]};
        }
        C* Y = smem_fft(bufa, bufb, 2 * nc, f.a1, tw1);
        for (int t = threadIdx.x; t < 2 * nc * Q1; t += blockDim.x) {
            const int cc = (int)qdiv((uint32_t)t, mQ1);   // pair * nc + line
            const int q = t - cc * Q1;
            const int pr = cc >= nc ? 1 : 0;
            const int c = cc - pr * nc;
            const int dst = (cpc == 1) ? q : (int)qdiv((uint32_t)q, mcpc);
            C* gg = cluster.map_shared_rank(gat, dst);
            gg[pr * gpair + (l0 + c0 + c) * cpc + (q - dst * cpc)] = Y[pad(cc * P1 + q)];
        }
        __syncthreads();
    }
    cp_async_wait_all();
    cluster.sync();
    // axis-0 pass: lines [pair 0: nc columns][pair 1: nc columns]
    SumAcc<float> acc0, acc1;
    for (int c0 = 0; c0 < nq; c0 += chunk) {
        const int nc = min(chunk, nq - c0);
        for (int t = threadIdx.x; t < 2 * nc * P0; t += blockDim.x) {
            const int cc = (int)qdiv((uint32_t)t, mP0);
            const int p = t - cc * P0;
            const int pr = cc >= nc ? 1 : 0;
            const int c = cc - pr * nc;
            int idx = p + off0;
            if (idx >= P0) idx -= P0;
            bufa[pad(t)] = (idx < S0) ? gat[pr * gpair + idx * cpc + c0 + c] : C{0.f, 0.f};
        }
        C* Y = smem_fft(bufa, bufb, 2 * nc, f.a0, tw0);
        for (int t = threadIdx.x; t < 2 * nc * P0; t += blockDim.x) {
            const int cc = (int)qdiv((uint32_t)t, mP0);
            const int w = t - cc * P0;
            const int pr = cc >= nc ? 1 : 0;
            const int c = cc - pr * nc;
            const int q = q0 + c0 + c;
            const float sv = spc[(c0 + c) * P0 + w] * float(half_weight(q, P1));
            const C y = Y[pad(t)];
            if (pr)
                acc1.add(sv * y.x, sv * y.y);
            else
                acc0.add(sv * y.x, sv * y.y);
        }
        __syncthreads();
    }
    double part0[2], part1[2];
    block_reduce_acc(acc0, part0);
    block_reduce_acc(acc1, part1);
    // every CTA receives every partial, so that each forms the same four sums
    // (same order, same rounding) and can run its own copy of the optimiser
    if (threadIdx.x == 0) {
        for (int r = 0; r < cs; ++r) {
            double* dst = cluster.map_shared_rank(cl_red, r);
            dst[4 * rank + 0] = part0[0];
            dst[4 * rank + 1] = part0[1];
            dst[4 * rank + 2] = part1[0];
            dst[4 * rank + 3] = part1[1];
        }
    }
    cluster.sync();
    if (threadIdx.x < 4) {
        double r = 0.0;
        for (int k = 0; k < cs; ++k) r += cl_red[4 * k + threadIdx.x];
        res4[threadIdx.x] = r * f.scale;
    }
}

// FP64 reciprocal and reciprocal square root from FP32 seeds refined by
// Newton-Raphson steps (each step squares the relative error): a few ulp of
// FP64 in a handful of FMAs, where the FP64 division and square root of
// this part are long dependent sequences.  Arguments outside the FP32 range
// take the FP64 operation.
__device__ __forceinline__ double rcp64(double x) {
    const double ax = fabs(x);
    if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
    double y = (double)__frcp_rn((float)x);
    y = fma(y, fma(-x, y, 1.0), y);
    y = fma(y, fma(-x, y, 1.0), y);
    return y;
}
__device__ __forceinline__ double rsqrt64(double x) {   // x > 0
    if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
    double y = (double)rsqrtf((float)x);
    const double hx = 0.5 * x;
    y = y * fma(-hx, y * y, 1.5);
    y = y * fma(-hx, y * y, 1.5);
    return y;
}
__device__ __forceinline__ double sqrt64(double x) { return x > 0.0 ? x * rsqrt64(x) : 0.0; }

// Optimiser state of one start (each CTA of its cluster holds a copy).  The
// search only compares FP32 evaluations and the value reported for its end
// point is recomputed at the FP64 bandwidth, so the quasi-Newton algebra is
// FP32 (FP64 arithmetic is slow on this part); the objective values and the
// parameters theta stay FP64.
struct SelOpt {
    float th[3], th_try[3];
    float g[3], dir[3], Binv[9];
    DFloat f;                 // objective at th, an unevaluated FP32 pair
    float step, slope;
    float dfp;                // decrease of the last accepted step (0: none since the last reset)
    float noise;              // resolution of the FP32 objective at th (0: not known)
    long long pts;            // lag route: half-box points evaluated
    double flops, bytes;      // FFT route: algorithmic work of the evaluations
    int iter, ls, done, evals, status, first;
    int fresh;   // the current direction comes from a reset (scaled steepest descent)
};

// a c - b^2 to about one FP32 ulp of the result however much the two
// products cancel (Kahan's 2 x 2 determinant with fused multiply-adds)
__device__ __forceinline__ float det2(float a, float b, float c) {
    const float w = b * b;
    const float e = fmaf(-b, b, w);   // w - b^2, exactly
    return fmaf(a, c, -w) + e;
}

// H = R R^T, R = [[e^t0, 0], [t1, e^t2]].
// Warp 0 of a CTA: trial point theta -> H, R and the work item; every
// lane returns false when H is outside the search domain (or needs a support
// beyond the cap / a size with no spectrum).  All lanes run the same
// straight-line FP32 code (lane s < nsig keeps covariance s), with the
// determinants in the compensated form of det2, which keeps a strongly
// correlated H's cancellation exact.  Every CTA of a cluster computes the
// same item from the same theta.  aux: determinant of H, work of the
// evaluation (lag route: half-box points; FFT route: flops), bytes.
__device__ bool sel_prepare(const SelectParams& p, const float* th, FusedItem<float>* it, float* Hs, float* Rs,
                            float* aux) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const float r00 = expf(th[0]), r11 = expf(th[2]), r10 = th[1];
    const float H[4] = {r00 * r00, r00 * r10, r10 * r00, fmaf(r10, r10, r11 * r11)};
    const float a = H[0], b = H[1], c = H[3];
    const float det = det2(a, b, c);
    // covariances: LSCV {2H, H}; SCV {2H + 2G, H + 2G, 2G}
    const int nsig = (p.method == 0) ? 2 : 3;
    const float gco = (p.method == 0) ? 0.f : 2.f;
    const float G[4] = {p.Gf[0], p.Gf[1], p.Gf[2], p.Gf[3]};
    const int sl = lane < nsig ? lane : 0;
    const float hco = (sl == 0) ? 2.f : (sl == 1 ? 1.f : 0.f);
    float iv0, iv1, iv3, nr;
    float xdv[12] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (p.method == 0) {
        float Ss[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) Ss[e] = hco * H[e];
        const float dts = det2(Ss[0], Ss[1], Ss[3]);
        const float rdt = __frcp_rn(dts);
        iv0 = Ss[3] * rdt;
        iv1 = -Ss[1] * rdt;
        iv3 = Ss[0] * rdt;
        nr = 0.15915494f * rsqrtf(dts);   // 1 / (2 pi sqrt(det))
    } else {
        // SCV: the kernel is evaluated relative to phi_{2G} (sel_grids), from
        // the exponent difference D_s and normaliser ratio rho_s of each
        // H-dependent Gaussian, which must be accurate well beyond FP32
        // because the kernel is much smaller than its terms.  With
        // Sigma_s = 2G + h_s H = 2G (I + h_s B), B = (2G)^-1 H, and the 2 x 2
        // identities det(I + h B) = 1 + h tr B + h^2 det B and
        // (I + h B)^-1 h B = (h B + h^2 det B I) / det(I + h B):
        //   Sigma_s^-1 - (2G)^-1 = -(h_s P + h_s^2 det(B) (2G)^-1) rho_s^2,
        //   rho_s = |Sigma_s|^-1/2 |2G|^1/2 = (1 + h_s tr B + h_s^2 det B)^-1/2,
        // P = (2G)^-1 H (2G)^-1: no difference of nearby values.  Lanes 0 and 1
        // (s = 0, 1) take it in FP32-pair arithmetic (about 44 bits) from the
        // FP32 trial H, which is exact there, with rho from an FP32 rsqrt and
        // one Newton step; lane 2 holds phi_{2G}.  No FP64 instruction: that
        // pipe is narrow on this part.  Entries in lag-index coordinates.
        iv0 = p.l2gj[0];
        iv1 = p.l2gj[1];
        iv3 = p.l2gj[2];
        nr = p.n2g;
        if (lane < 2) {
            const float hs = (lane == 0) ? 2.f : 1.f;
            const float h00 = H[0], h01 = H[1], h11 = H[3];
            const DFloat L00{p.l2gh[0], p.l2gl[0]}, L01{p.l2gh[1], p.l2gl[1]}, L11{p.l2gh[2], p.l2gl[2]};
            const DFloat m00 = df_add(df_mulf(L00, h00), df_mulf(L01, h01));
            const DFloat m01 = df_add(df_mulf(L00, h01), df_mulf(L01, h11));
            const DFloat m10 = df_add(df_mulf(L01, h00), df_mulf(L11, h01));
            const DFloat m11 = df_add(df_mulf(L01, h01), df_mulf(L11, h11));
            const DFloat P[3] = {df_add(df_mul(m00, L00), df_mul(m01, L01)), df_add(df_mul(m00, L01), df_mul(m01, L11)),
                                 df_add(df_mul(m10, L01), df_mul(m11, L11))};
            const DFloat q01 = df_prod(h01, h01);
            const DFloat detH = df_add(df_prod(h00, h11), DFloat{-q01.h, -q01.l});
            const DFloat hh = df_mulf(df_mul(DFloat{p.dl2gh, p.dl2gl}, detH), hs * hs);   // h_s^2 det B
            const DFloat xg = df_add(df_add(df_mulf(df_add(m00, m11), hs), hh), DFloat{1.f, 0.f});
            // rho = xg^-1/2: y + y (1 - xg y^2) / 2 from the FP32 estimate y
            const float y = rsqrtf(xg.h);
            const DFloat xy2 = df_mul(xg, df_prod(y, y));
            const DFloat rho = df_two_sum(y, 0.5f * y * ((1.f - xy2.h) - xy2.l));
            const DFloat r2 = df_mul(rho, rho);
            const DFloat Ls[3] = {L00, L01, L11};
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const DFloat num = df_add(df_mulf(P[e], hs), df_mul(hh, Ls[e]));
                const DFloat De = df_mul(df_mul(num, r2), DFloat{p.ddh[e], p.ddl[e]});
                xdv[e] = -De.h;
                xdv[3 + e] = -De.l;
            }
            const DFloat rm1 = df_add(rho, DFloat{-1.f, 0.f});
            xdv[6] = rho.h;
            xdv[7] = rho.l;
            xdv[8] = rm1.h;
            xdv[9] = rm1.l;
            iv0 += xdv[0];
            iv1 += xdv[1];
            iv3 += xdv[2];
        }
    }
    // supports from lambda_max of H (LSCV, paper rule), 2H (LSCV widest) or 2H + 2G (SCV)
    const float bs = (p.method == 1 || p.widest) ? 2.f : 1.f;
    float B[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) B[e] = fmaf(bs, H[e], gco * G[e]);
    const float tr = 0.5f * (B[0] + B[3]), dd = 0.5f * (B[0] - B[3]);
    const float sq = sqrtf(fabsf(tr + sqrtf(fmaf(dd, dd, B[1] * B[1]))));
    const float tau = p.tauf;
    float v0 = ceilf(tau * sq * p.rd0f);
    float v1 = ceilf(tau * sq * p.rd1f);
    v0 = fminf(fmaxf(v0, 1.f), (float)(p.M0 - 1));
    v1 = fminf(fmaxf(v1, 1.f), (float)(p.M1 - 1));
    const int L0 = (int)v0, L1 = (int)v1;
    // the bandwidth is at least half a bin wide along each axis
    const float d0 = p.d0f, d1 = p.d1f;
    const bool inside = a > 0.f && det > 0.f && a >= 0.25f * d0 * d0 && c >= 0.25f * d1 * d1 && !(v0 != v0) &&
                        !(v1 != v1);
    if (!inside || L0 > p.Lcap || L1 > p.Lcap1) return false;
    // FFT route: the count spectrum of the padded size for (L0, L1)
    int si = -1;
    const int P0 = p.acorr ? 0 : p.ptab0[L0], P1 = p.acorr ? 0 : p.ptab1[L1];
    for (int i0 = 0; !p.acorr && i0 < p.nspec && si < 0; i0 += 32) {
        const int i = i0 + lane;
        const unsigned m = __ballot_sync(FULL, i < p.nspec && p.specs[i].P0 == P0 && p.specs[i].P1 == P1);
        if (m) si = i0 + __ffs(m) - 1;
    }
    if (!p.acorr && si < 0) {
        if (lane == 0) atomicOr(p.errflag, 2);
        return false;
    }
    // the work item (one: the four grids of a bandwidth are evaluated
    // together), its stores spread over lanes: lanes 0..2 the covariance
    // rows (lanes 0 and 1 also SCV's exponent differences), lane 3 the
    // header, lane 4 the bandwidth and its factor (the caller's barrier
    // publishes them)
    if (lane < MAXSIG) {
        const bool on = lane < nsig;
        const float iv[4] = {on ? iv0 : 0.f, on ? iv1 : 0.f, on ? iv1 : 0.f, on ? iv3 : 0.f};
#pragma unroll
        for (int e = 0; e < 4; ++e) it[0].laml[lane][e] = iv[e];
        it[0].nrm[lane] = on ? nr : 0.f;
        if (lane < 2 && p.method == 1)
#pragma unroll
            for (int e = 0; e < 12; ++e) it[0].xd[lane][e] = xdv[e];
    }
    if (lane == 3) {
        FusedItem<float>& f = it[0];
        f.S0 = 2 * L0 + 1;
        f.S1 = 2 * L1 + 1;
        f.off0 = L0;
        f.off1 = L1;
        f.nsig = nsig;
        f.pad_ = 0;
        f.delta0 = p.delta0;
        f.delta1 = p.delta1;
        if (p.acorr) {   // lag domain: n^-2, no transform
            f.spec = nullptr;
            f.scale = p.inv_n2;
        } else {
            const SelSpec& sp = p.specs[si];
            f.a0 = sp.a0;
            f.a1 = sp.a1;
            f.spec = sp.spec;
            f.scale = sp.scale;
        }
    }
    // (both routes evaluate the four grids with sel_grids: no dense weights)
    if (lane == 4) {
        for (int e = 0; e < 4; ++e) Hs[e] = H[e];
        Rs[0] = r00;
        Rs[1] = r10;
        Rs[2] = r11;
        aux[0] = det;
        if (p.acorr) {   // half-box points (exact in FP32 below 2^24)
            aux[1] = (float)((L0 + 1) * (2 * L1 + 1));
            aux[2] = 0.f;
        } else {
            const SelSpec& sp = p.specs[si];
            aux[1] = (float)(sp.fl_fix + (double)(2 * L0 + 1) * sp.fl_line);
            aux[2] = (float)sp.by;
        }
    }
    return true;
}

// objective, gradient in H (tied convention) -> value and theta-gradient
// (FP32 algebra; the value is the FP32 pair sum of the device sum r[0] and
// the closed-form term; r[1..3]: the sums of the three derivative grids)
__device__ void sel_assemble(const SelectParams& p, const float* H, const float* Rm, const DFloat* r, float det,
                             DFloat* f, float* gt, float* gH = nullptr, float* fsc = nullptr) {
    const float rdet = __frcp_rn(det);
    const float rsd = rsqrtf(det);   // |H|^-1/2
    const float rn = p.inv_nf;
    const float hi00 = H[3] * rdet, hi01 = -H[1] * rdet, hi11 = H[0] * rdet;
    const float r1 = r[1].h + r[1].l, r2 = r[2].h + r[2].l, r3 = r[3].h + r[3].l;
    float g00, g01, g11;
    if (p.method == 0) {
        const float k0 = 0.15915494f * rsd;   // K_H(0) = (2 pi)^-1 |H|^-1/2, Eq. 11
        const float c0 = 2.f * rn;
        *f = df_add(r[0], DFloat{c0 * k0, 0.f});
        if (fsc) *fsc = r[4].h + c0 * k0;   // magnitude of the summed terms
        g00 = r1 + c0 * (-0.5f * k0 * hi00);
        g01 = r2 + c0 * 2.f * (-0.5f * k0 * hi01);
        g11 = r3 + c0 * (-0.5f * k0 * hi11);
    } else {
        // the derivative grids were summed in lag-index coordinates
        const float rk = 0.07957747f * rsd;   // (4 pi)^-1 |H|^-1/2
        *f = df_add(r[0], DFloat{rk * rn, 0.f});
        if (fsc) *fsc = r[4].h + rk * rn;
        g00 = fmaf(r1, p.gsc[0], (-0.5f * rk * hi00) * rn);
        g01 = fmaf(r2, p.gsc[1], 2.f * (-0.5f * rk * hi01) * rn);
        g11 = fmaf(r3, p.gsc[2], (-0.5f * rk * hi11) * rn);
    }
    if (gH) {
        gH[0] = g00;
        gH[1] = g01;
        gH[2] = g11;
    }
    // dF/dR = 2 G_ind R (G_ind off-diagonal = g01 / 2), chain rule to theta
    const float G00 = g00, G01 = 0.5f * g01, G11 = g11;
    const float R00 = (float)Rm[0], R10 = (float)Rm[1], R11 = (float)Rm[2];
    const float d00 = 2.f * (G00 * R00 + G01 * R10);
    const float d10 = 2.f * (G01 * R00 + G11 * R10);
    const float d11 = 2.f * (G11 * R11);
    gt[0] = d00 * R00;
    gt[1] = d10;
    gt[2] = d11 * R11;
}

__device__ void sel_new_direction(SelOpt& s) {
    for (int i = 0; i < 3; ++i) {
        float v = 0.f;
        for (int j = 0; j < 3; ++j) v -= s.Binv[i * 3 + j] * s.g[j];
        s.dir[i] = v;
    }
    s.slope = s.dir[0] * s.g[0] + s.dir[1] * s.g[1] + s.dir[2] * s.g[2];
    if (!(s.slope < 0.f)) {
        const float gn = fmaxf(fabsf(s.g[0]), fmaxf(fabsf(s.g[1]), fabsf(s.g[2])));
        const float sc = (gn > 0.f) ? 0.1f * __frcp_rn(gn) : 1.f;
        for (int i = 0; i < 9; ++i) s.Binv[i] = 0.f;
        for (int i = 0; i < 3; ++i) {
            s.Binv[i * 4] = sc;
            s.dir[i] = -sc * s.g[i];
        }
        s.slope = s.dir[0] * s.g[0] + s.dir[1] * s.g[1] + s.dir[2] * s.g[2];
    }
    const float dm = fmaxf(fabsf(s.dir[0]), fmaxf(fabsf(s.dir[1]), fabsf(s.dir[2])));
    if (dm > 1.f) {
        const float r = __frcp_rn(dm);
        for (int i = 0; i < 3; ++i) s.dir[i] *= r;
        s.slope *= r;
    }
    // first trial step: the minimiser of the quadratic that repeats the last
    // accepted decrease along the new direction, 1.01 x 2 (f_k - f_{k-1}) /
    // slope, at most 1 (the unit quasi-Newton step)
    float a0 = 1.f;
    if (s.dfp < 0.f) {
        const float q = 2.02f * s.dfp * __frcp_rn(s.slope);
        if (q > 0.f) a0 = fminf(1.f, q);
    }
    s.step = a0;
    s.ls = 0;
    for (int i = 0; i < 3; ++i) s.th_try[i] = s.th[i] + s.step * s.dir[i];
    if (-a0 * s.slope <= s.noise) s.done = 1;   // nothing left to resolve along this direction
}

// sums of one lag-domain evaluation: the four grids and the magnitude of the
// objective's terms
constexpr int SEL_NSUM = 5;

// Backtracking: a rejected trial step is replaced by the minimiser of the
// quadratic through f(0), the slope f'(0) and f(step), kept within
// [0.1, 0.5] of the step (safeguarded interpolation); a trial point outside
// the search domain halves the step.  The line search gives up after
// kMaxBacktracks rejections, or as soon as the next trial point would move
// theta by less than kStepFloor in every coordinate (a relative change of
// about 2e-5 in H), which the FP32 objective cannot resolve: the binned
// objective also steps where a support L_k changes with H (Eq. 26), and a
// sufficient-decrease test at smaller steps only measures those steps.
constexpr int kMaxBacktracks = 12;
constexpr float kStepFloor = 1e-5f;
// Resolution of an FP32 objective value relative to the magnitude S of its
// summed terms (measured against the FP64 oracle: errors up to about
// 6e-7 S).  Where S is known (lag route), a search also stops when an accepted
// step, or the first-order decrease predicted for the next trial step, is
// below kResolution S: such differences are rounding, not descent.
constexpr float kResolution = 2e-7f;

// consume the evaluation (fn, gn) of the trial point th_try.  The value is
// an FP32 pair: the difference of two nearby values (Sterbenz: the leading
// parts subtract exactly) keeps about 14 digits.
__device__ void sel_update(SelOpt& s, DFloat fn, const float* gn, int max_iter, float fscale = 0.f) {
    if (s.first) {
        s.first = 0;
        s.f = fn;
        s.noise = kResolution * fscale;
        for (int i = 0; i < 3; ++i) {
            s.th[i] = s.th_try[i];
            s.g[i] = gn[i];
        }
        if (!isfinite(fn.h)) {
            s.done = 1;
            s.status = 2;
            return;
        }
        const float gm = fmaxf(fabsf(gn[0]), fmaxf(fabsf(gn[1]), fabsf(gn[2])));
        const float sc = (gm > 0.f) ? 0.1f * __frcp_rn(gm) : 1.f;
        for (int i = 0; i < 9; ++i) s.Binv[i] = 0.f;
        for (int i = 0; i < 3; ++i) s.Binv[i * 4] = sc;
        if (gm == 0.f) {
            s.done = 1;
            return;
        }
        s.fresh = 1;
        s.dfp = 0.f;
        sel_new_direction(s);
        return;
    }
    const float df = (fn.h - s.f.h) + (fn.l - s.f.l);   // fn - f
    if (isfinite(fn.h) && df <= 1e-4f * (s.step * s.slope)) {
        float sv[3], yv[3], sy = 0.f;
        for (int i = 0; i < 3; ++i) {
            sv[i] = s.th_try[i] - s.th[i];
            yv[i] = gn[i] - s.g[i];
            sy += sv[i] * yv[i];
        }
        if (sy > 1e-30f) {
            float By[3], yBy = 0.f;
            for (int i = 0; i < 3; ++i) {
                By[i] = 0.f;
                for (int j = 0; j < 3; ++j) By[i] += s.Binv[i * 3 + j] * yv[j];
                yBy += yv[i] * By[i];
            }
            const float rsy = __frcp_rn(sy);
            const float c1 = (sy + yBy) * rsy * rsy;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    s.Binv[i * 3 + j] += c1 * sv[i] * sv[j] - (By[i] * sv[j] + sv[i] * By[j]) * rsy;
        }
        float gm = 0.f, tn = 0.f;
        for (int i = 0; i < 3; ++i) {
            s.th[i] = s.th_try[i];
            s.g[i] = gn[i];
            gm = fmaxf(gm, fabsf(gn[i]));
            tn = fmaxf(tn, fabsf(sv[i]));
        }
        s.f = fn;
        s.dfp = df;
        s.noise = kResolution * fscale;
        s.iter++;
        if (s.iter >= max_iter) {
            s.done = 1;
            s.status = 1;
        } else if (fabsf(df) <= 1e-12f * fabsf(fn.h) + 1e-30f || -df <= s.noise || tn < 1e-10f ||
                   gm < 1e-12f * (fabsf(fn.h) + 1e-30f)) {
            s.done = 1;
        } else {
            s.fresh = 0;
            sel_new_direction(s);
        }
    } else {
        float nstep = 0.5f * s.step;
        if (isfinite(fn.h)) {
            const float pred = s.step * s.slope;   // < 0
            const float den = df - pred;           // > 0 after a failed sufficient-decrease test
            if (den > 0.f) nstep = fminf(fmaxf(-0.5f * pred * s.step * __frcp_rn(den), 0.1f * s.step), 0.5f * s.step);
        }
        s.step = nstep;
        s.ls++;
        const float dm = fmaxf(fabsf(s.dir[0]), fmaxf(fabsf(s.dir[1]), fabsf(s.dir[2])));
        const bool give_up = s.ls > kMaxBacktracks || s.step * dm < kStepFloor || -s.step * s.slope <= s.noise;
        if (give_up && !s.fresh) {
            // restart: the quasi-Newton model failed here; scaled steepest descent once
            const float gm = fmaxf(fabsf(s.g[0]), fmaxf(fabsf(s.g[1]), fabsf(s.g[2])));
            const float sc = (gm > 0.f) ? 0.1f * __frcp_rn(gm) : 1.f;
            for (int i = 0; i < 9; ++i) s.Binv[i] = 0.f;
            for (int i = 0; i < 3; ++i) s.Binv[i * 4] = sc;
            s.fresh = 1;
            s.dfp = 0.f;
            sel_new_direction(s);
        } else if (give_up) {
            s.done = 1;
        } else {
            for (int i = 0; i < 3; ++i) s.th_try[i] = s.th[i] + s.step * s.dir[i];
        }
    }
}

// One evaluation of the search into the caller's record (thread 0; only
// when recording is on and the start has slots left).
__device__ __forceinline__ void sel_record(const SelectParams& p, int start, int e, const float* H, int L0, int L1,
                                          DFloat f, const float* gH) {
    if (!p.rec || e >= p.rec_cap) return;
    double* r = p.rec + ((size_t)start * p.rec_cap + e) * SEL_REC;
    r[0] = start;
    r[1] = e;
    r[2] = p.method;
    r[3] = H[0];
    r[4] = H[1];
    r[5] = H[3];
    r[6] = L0;
    r[7] = L1;
    r[8] = (double)f.h + (double)f.l;
    r[9] = gH[0];
    r[10] = gH[1];
    r[11] = gH[2];
}

__global__ void __launch_bounds__(256) k_select2d(SelectParams p, SelStart* __restrict__ starts,
                                                  const float2* __restrict__ twpool) {
    using C = float2;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double cl_red[64];
    __shared__ double res[2][2];
    __shared__ FusedItem<float> items[1];
    __shared__ SelOpt opt;
    __shared__ int ctl[2];              // [valid, done] of this round
    __shared__ float Hs[4], Rs[3], aux[3];
    C* gat = reinterpret_cast<C*>(smem_raw);
    float* spc = reinterpret_cast<float*>(gat + p.gat_elems);
    C* tw1 = reinterpret_cast<C*>(spc + p.spc_elems);
    C* tw0 = tw1 + p.pmax;
    C* bufa = tw0 + p.pmax;
    C* bufb = bufa + padded_cap(p.cap);
    const int rank = (int)cluster.block_rank();
    const int start = blockIdx.x / p.cs;
    if (threadIdx.x == 0) {
        const SelStart& st = starts[start];
        for (int i = 0; i < 3; ++i) opt.th_try[i] = (float)st.th[i];
        opt.first = 1;
        opt.done = 0;
        opt.iter = 0;
        opt.evals = 0;
        opt.status = 0;
        opt.f = DFloat{INFINITY, 0.f};
        opt.pts = 0;
        opt.flops = 0.0;
        opt.bytes = 0.0;
        opt.fresh = 0;
        opt.dfp = 0.f;
        opt.noise = 0.f;
    }
    __syncthreads();
    const int max_rounds = 40 * p.max_iter + 2;
    for (int round = 0; round < max_rounds; ++round) {
        if (threadIdx.x < 32) {
            const int dn = opt.done;
            const bool v = dn ? false : sel_prepare(p, opt.th_try, items, Hs, Rs, aux);
            if (threadIdx.x == 0) {
                ctl[0] = v ? 1 : 0;
                ctl[1] = dn;
            }
        }
        __syncthreads();
        const int valid = ctl[0], done = ctl[1];
        if (done) break;
        if (valid) {
            if (p.method == 0)
                sel_eval2<0>(cluster, items[0], p.cs, rank, p.chunk, gat, spc, tw1, tw0, bufa, bufb, twpool,
                             cl_red, &res[0][0]);
            else
                sel_eval2<1>(cluster, items[0], p.cs, rank, p.chunk, gat, spc, tw1, tw0, bufa, bufb, twpool,
                             cl_red, &res[0][0]);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            DFloat fn{INFINITY, 0.f};
            float gt[3] = {0.f, 0.f, 0.f};
            if (valid) {
                // the cluster sums arrive in FP64: split each into an FP32 pair
                DFloat r[4];
                const double rv[4] = {res[0][0], res[0][1], res[1][0], res[1][1]};
                for (int e = 0; e < 4; ++e) {
                    const float h = (float)rv[e];
                    r[e] = DFloat{h, (float)(rv[e] - (double)h)};
                }
                float gH[3];
                sel_assemble(p, Hs, Rs, r, aux[0], &fn, gt, gH);
                if (rank == 0) sel_record(p, start, opt.evals, Hs, items[0].off0, items[0].off1, fn, gH);
                opt.evals++;
                opt.flops += (double)aux[1];
                opt.bytes += (double)aux[2];
            }
            sel_update(opt, fn, gt, p.max_iter);
        }
        __syncthreads();
    }
    if (rank == 0 && threadIdx.x == 0) {
        SelStart& st = starts[start];
        for (int i = 0; i < 3; ++i) st.th[i] = opt.th[i];
        st.f = (double)opt.f.h + (double)opt.f.l;
        st.evals = opt.evals;
        st.iters = opt.iter;
        st.status = opt.done ? opt.status : 1;
        st.flops = opt.flops;
        st.bytes = opt.bytes;
    }
}

// One bandwidth of the search in the lag domain by the CS CTAs of a cluster
// (CS = 1: one CTA): the half box j_0 in [0, L_0], |j_1| <= L_1 (j_0
// fastest, so that neighbouring threads read neighbouring a_j), weights
// 2 / 1 / 0, compensated sums of the four grids and of |grid 0| (the
// magnitude of the objective's summed terms: its FP32 resolution scale).
// With CS > 1 the points are dealt out over the cluster's threads; every
// CTA sends its partial sums to all CTAs (distributed shared memory, clp =
// this round's buffer, [CS][NSUM]), and after one cluster barrier each sums
// them in rank order, so that every CTA holds the same totals.  Lanes
// 0..NSUM-1 of warp 0 write the NSUM scaled totals to res4 (shared; the
// caller's barrier publishes them).  The CTA has at least NSUM warps.
template <int METHOD, int CS>
__device__ __forceinline__ void sel_eval_lag(const FusedItem<float>& f, const float* __restrict__ acorr, int A0,
                                             int A1, float d0f, float d1f, DFloat scale, DFloat* res4, DFloat* clp,
                                             int rank) {
    const int L0 = f.off0, L1 = f.off1;
    const int n0 = L0 + 1;
    const int total = n0 * (2 * L1 + 1);
    const uint32_t mn0 = magic_of((uint32_t)max(n0, 2));
    // the multiply-high quotient is exact while t n0 < 2^32 for every t <
    // total (large boxes on grids beyond ~1500 nodes divide plainly)
    const bool fastq = (unsigned long long)total * (unsigned long long)n0 < (1ULL << 32);
    const float d0 = d0f, d1 = d1f;
    // a thread holds a few points: plain FP32 sums there and across its warp
    // (the search compares values to FP32 accuracy; the reported value is
    // recomputed), compensated sums across the warps
    constexpr int NS = SEL_NSUM;
    float s4[NS] = {0.f, 0.f, 0.f, 0.f, 0.f};
    // warp w of CTA r takes the 32-point runs w CS + r (+ k CS warps): the
    // CTAs of a cluster get equal shares, and a warp past the end of the box
    // skips the shuffles below
    const int wi = threadIdx.x >> 5, li = threadIdx.x & 31;
    const bool wact = (wi * CS + rank) * 32 < total;
    for (int t = (wi * CS + rank) * 32 + li; t < total; t += CS * (int)blockDim.x) {
        const int q = (n0 == 1) ? t : (fastq ? (int)qdiv((uint32_t)t, mn0) : t / n0);
        const int j0 = t - q * n0;
        const int j1 = q - L1;
        const int wt = (j0 > 0 || j1 > 0) ? 2 : (j1 == 0 ? 1 : 0);
        if (!wt) continue;
        const float av = acorr[(j1 + A1) * (A0 + 1) + j0];
        float v[4];
        sel_grids<METHOD>(f, j0, j1, d0, d1, v);
        const float wa = (float)wt * av;
#pragma unroll
        for (int e = 0; e < 4; ++e) s4[e] = fmaf(wa, v[e], s4[e]);
        s4[4] = fmaf(wa, fabsf(v[0]), s4[4]);
    }
    __shared__ float red4[NS][32];
    if (wact)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int e = 0; e < NS; ++e) s4[e] += __shfl_down_sync(0xffffffffu, s4[e], o);
    if (li == 0)
#pragma unroll
        for (int e = 0; e < NS; ++e) red4[e][wi] = s4[e];
    __syncthreads();
    // warp e (e < NS; the CTA has at least NS warps) sums value e over the
    // warps as FP32 pairs, in a fixed tree: the NS sums run on NS warps side
    // by side instead of interleaved on one
    __shared__ DFloat tot[NS];
    if (wi < NS) {
        const int e = wi;
        const int nw = (blockDim.x + 31) >> 5;
        DFloat v{(li < nw) ? red4[e][li] : 0.f, 0.f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const DFloat t{__shfl_down_sync(0xffffffffu, v.h, o), __shfl_down_sync(0xffffffffu, v.l, o)};
            v = df_add(v, t);
        }
        if constexpr (CS > 1) {
            // lane r < CS sends this CTA's total (held by lane 0) to CTA r
            v = DFloat{__shfl_sync(0xffffffffu, v.h, 0), __shfl_sync(0xffffffffu, v.l, 0)};
            if (li < CS) cg::this_cluster().map_shared_rank(clp, li)[rank * NS + e] = v;
        } else {
            if (li == 0) tot[e] = v;
        }
    }
    if constexpr (CS > 1)
        cg::this_cluster().sync();
    else
        __syncthreads();
    if (wi == 0 && li < NS) {
        // lane e: value e summed over the CTAs in rank order, times n^-2 as
        // FP32 pairs
        const int e = li;
        DFloat v;
        if constexpr (CS > 1) {
            v = clp[e];
#pragma unroll
            for (int r = 1; r < CS; ++r) v = df_add(v, clp[r * NS + e]);
        } else {
            v = tot[e];
        }
        const float ph = v.h * scale.h;
        const float pl = fmaf(v.h, scale.h, -ph) + fmaf(v.h, scale.l, v.l * scale.h);
        const float h = ph + pl;
        res4[e] = DFloat{h, pl - (h - ph)};
    }
}

// One start's whole quasi-Newton search with lag-domain evaluations against
// the count autocorrelation (staged in shared memory, or read from the
// L2-resident FP32 copy), by one CTA or a cluster of CS CTAs.  Every CTA of
// a cluster runs its own copy of the optimiser state (in the caller's
// shared memory) on the same totals, so all take the same branches and meet
// at the same cluster barriers; rank 0 writes the record and the result.
template <int CS>
__device__ __forceinline__ void sel_search_lag(const SelectParams& p, SelStart* __restrict__ starts, int start,
                                               const float* acorr, DFloat* res, FusedItem<float>* items,
                                               SelOpt& opt, int* ctl, float* Hs, float* Rs, float* aux,
                                               DFloat* clp /* [2][CS][SEL_NSUM] */, int rank) {
    if (threadIdx.x == 0) {
        const SelStart& st = starts[start];
        for (int i = 0; i < 3; ++i) opt.th_try[i] = (float)st.th[i];
        opt.first = 1;
        opt.done = 0;
        opt.iter = 0;
        opt.evals = 0;
        opt.status = 0;
        opt.f = DFloat{INFINITY, 0.f};
        opt.pts = 0;
        opt.flops = 0.0;
        opt.bytes = 0.0;
        opt.fresh = 0;
        opt.dfp = 0.f;
        opt.noise = 0.f;
    }
    __syncthreads();
    const int max_rounds = 40 * p.max_iter + 2;
    for (int round = 0; round < max_rounds; ++round) {
        if (threadIdx.x < 32) {
            const int dn = opt.done;
            const bool v = dn ? false : sel_prepare(p, opt.th_try, items, Hs, Rs, aux);
            if (threadIdx.x == 0) {
                ctl[0] = v ? 1 : 0;
                ctl[1] = dn;
            }
        }
        __syncthreads();
        const int valid = ctl[0], done = ctl[1];
        if (done) break;
        if (valid) {
            // partial sums alternate between two buffers, so that a CTA ahead
            // by a round never overwrites totals another CTA is still reading
            DFloat* cb = clp + (round & 1) * (CS * SEL_NSUM);
            const DFloat sc{p.inv_n2h, p.inv_n2l};
            if (p.method == 0)
                sel_eval_lag<0, CS>(items[0], acorr, p.A0, p.A1, p.d0f, p.d1f, sc, res, cb, rank);
            else
                sel_eval_lag<1, CS>(items[0], acorr, p.A0, p.A1, p.d0f, p.d1f, sc, res, cb, rank);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            DFloat fn{INFINITY, 0.f};
            float gt[3] = {0.f, 0.f, 0.f};
            float fsc = 0.f;
            if (valid) {
                float gH[3];
                sel_assemble(p, Hs, Rs, res, aux[0], &fn, gt, gH, &fsc);
                if (rank == 0) sel_record(p, start, opt.evals, Hs, items[0].off0, items[0].off1, fn, gH);
                opt.evals++;
                opt.pts += (long long)aux[1];
            }
            sel_update(opt, fn, gt, p.max_iter, fsc);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && rank == 0) {
        // per half-box point and covariance: a quadratic form (8 flops) and
        // four six-term weighted sums (48); 4 bytes of autocorrelation
        const double nsig = (p.method == 0) ? 2.0 : 3.0;
        SelStart& st = starts[start];
        for (int i = 0; i < 3; ++i) st.th[i] = opt.th[i];
        st.f = (double)opt.f.h + (double)opt.f.l;
        st.evals = opt.evals;
        st.iters = opt.iter;
        st.status = opt.done ? opt.status : 1;
        st.flops = (double)opt.pts * nsig * 56.0;
        st.bytes = (double)opt.pts * sizeof(float);
    }
}

// Two searches on one dataset in one launch: starts [0, nfirst) run
// criterion p, the rest criterion q (the same autocorrelation box).  A
// single search passes q = p.  Start s runs on CTAs [s CS, (s + 1) CS), one
// cluster.
template <int CS>
__global__ void __launch_bounds__(1024) k_select2d_lag(SelectParams p, SelectParams q, int nfirst,
                                                       SelStart* __restrict__ starts, int stage) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ DFloat res[SEL_NSUM];
    __shared__ FusedItem<float> items[1];
    __shared__ SelOpt opt;
    __shared__ int ctl[2];
    __shared__ float Hs[4], Rs[3], aux[3];
    __shared__ DFloat clp[2 * CS * SEL_NSUM];
    const int start = (int)blockIdx.x / CS;
    const int rank = (CS > 1) ? (int)cg::this_cluster().block_rank() : 0;
    // the autocorrelation box is fixed for the whole search: staged once in
    // shared memory when it fits (stage != 0)
    const float* acorr = p.acorr;
    if (stage) {
        float* sa = reinterpret_cast<float*>(smem_raw);
        const int nbox = (p.A0 + 1) * (2 * p.A1 + 1);
        for (int t = threadIdx.x; t < nbox; t += blockDim.x) sa[t] = p.acorr[t];
        acorr = sa;
    }
    if (start < nfirst)
        sel_search_lag<CS>(p, starts, start, acorr, res, items, opt, ctl, Hs, Rs, aux, clp, rank);
    else
        sel_search_lag<CS>(q, starts, start, acorr, res, items, opt, ctl, Hs, Rs, aux, clp, rank);
    // no CTA leaves while another may still write into its shared memory
    if constexpr (CS > 1) cg::this_cluster().sync();
}

// Cluster size for a launch: the largest of 4, 2 whose clusters are all
// co-resident (one wave), else one CTA per start.  Queried once per device
// and shared-memory size.
static int select2d_lag_cs(int nstarts, size_t sm) {
    static std::mutex mu;
    static std::map<std::tuple<int, size_t, int>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(mu);
    for (int cs : {4, 2}) {
        const auto key = std::make_tuple(dev, sm, cs);
        auto it = cache.find(key);
        if (it == cache.end()) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            cfg.gridDim = dim3((unsigned)cs, 1, 1);
            cfg.blockDim = dim3(1024, 1, 1);
            cfg.dynamicSmemBytes = sm;
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = (unsigned)cs;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int n = 0;
            const void* f = (cs == 4) ? (const void*)k_select2d_lag<4> : (const void*)k_select2d_lag<2>;
            if (cudaOccupancyMaxActiveClusters(&n, f, &cfg) != cudaSuccess) {
                cudaGetLastError();
                n = 0;
            }
            it = cache.emplace(key, n).first;
        }
        if (it->second >= nstarts) return cs;
    }
    return 1;
}

template <int CS>
static cudaError_t launch_select2d_lag_cs(const SelectParams& prm, const SelectParams& prm2, int nfirst,
                                          SelStart* starts, int nstarts, size_t sm, int stage, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)(nstarts * CS), 1, 1);
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_select2d_lag<CS>, prm, prm2, nfirst, starts, stage);
}

cudaError_t launch_select2d_lag(const SelectParams& prm, const SelectParams& prm2, int nfirst, SelStart* starts,
                                int nstarts, cudaStream_t st) {
    // dynamic shared memory for the staged box: up to `limit` on top of the
    // kernel's static shared memory (within the limit prepare_kernels set)
    const size_t box = sizeof(float) * (size_t)(prm.A0 + 1) * (size_t)(2 * prm.A1 + 1);
    const size_t limit = 200 * 1024;
    const int stage = box <= limit ? 1 : 0;
    const size_t sm = stage ? box : 0;
    const int cs = select2d_lag_cs(nstarts, sm);
    if (cs == 4) return launch_select2d_lag_cs<4>(prm, prm2, nfirst, starts, nstarts, sm, stage, st);
    if (cs == 2) return launch_select2d_lag_cs<2>(prm, prm2, nfirst, starts, nstarts, sm, stage, st);
    k_select2d_lag<1><<<nstarts, 1024, sm, st>>>(prm, prm2, nfirst, starts, stage);
    return cudaGetLastError();
}

static size_t select2d_smem(const SelectParams& prm) {
    return sizeof(float2) * (size_t)(prm.gat_elems + 2 * prm.pmax + 2 * padded_cap(prm.cap)) +
           sizeof(float) * (size_t)prm.spc_elems;
}

static cudaError_t select2d_config(const SelectParams& prm, int nstarts, cudaStream_t st, cudaLaunchConfig_t& cfg,
                                   cudaLaunchAttribute* attr) {
    const size_t sm = select2d_smem(prm);
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3((unsigned)(nstarts * prm.cs), 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)prm.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaSuccess;
}

cudaError_t launch_select2d(const SelectParams& prm, SelStart* starts, int nstarts, const float2* twpool,
                            cudaStream_t st) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e = select2d_config(prm, nstarts, st, cfg, attr);
    if (e != cudaSuccess) return e;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_select2d, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return cudaErrorNotSupported;
    }
    return cudaLaunchKernelEx(&cfg, k_select2d, prm, starts, twpool);
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
    k_stage_a<real><<<grid, 256, sm, st>>>(items, tiles, ntiles, cap, scratch, twpool, partial);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_mid(const Item<real>* items, const Tile* tiles, int ntiles, int axis, int pmax, int cap,
                       typename Cpx<real>::T* scratch, const typename Cpx<real>::T* twpool, int grid,
                       cudaStream_t st) {
    const size_t sm = smem_bytes<real>(cap, pmax);
    k_mid<real><<<grid, 256, sm, st>>>(items, tiles, ntiles, axis, cap, scratch, twpool);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_final(const Item<real>* items, const Tile* tiles, int ntiles, int pmax, int cap,
                         typename Cpx<real>::T* scratch, const typename Cpx<real>::T* twpool, double* partial,
                         int grid, cudaStream_t st) {
    // ping-pong buffers, twiddles, then the staged spectrum rows (cap reals)
    const size_t sm = smem_bytes<real>(cap, pmax) + sizeof(real) * (size_t)cap;
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
        // clusters above the portable size must be schedulable with this
        // shared-memory footprint (checked once per device, cluster size and
        // footprint; the cache is shared by every context of the process)
        static std::mutex mu;
        static std::map<std::tuple<int, int, size_t>, bool> fits;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorNotSupported;
        std::lock_guard<std::mutex> lk(mu);
        const auto key = std::make_tuple(dev, cs, sm);
        auto it = fits.find(key);
        if (it == fits.end()) {
            int nclusters = 0;
            bool ok = cudaOccupancyMaxActiveClusters(&nclusters, k_fused2d<real, R>, &cfg) == cudaSuccess && nclusters >= 1;
            if (!ok) cudaGetLastError();
            it = fits.emplace(key, ok).first;
        }
        if (!it->second) return cudaErrorNotSupported;
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

// Every kernel that may take more than the default 48 KB of dynamic shared
// memory gets the device's opt-in maximum (less its static shared memory),
// and the cluster kernels may use non-portable cluster sizes.  Set once per
// device before any launch -- at context creation and by the first
// allocation-free call -- so that no launch sets (or could lower) a limit
// another thread's launch relies on.  Idempotent.
cudaError_t prepare_kernels() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    auto raise = [&](const void* f) -> cudaError_t {
        cudaFuncAttributes fa;
        cudaError_t r = cudaFuncGetAttributes(&fa, f);
        if (r != cudaSuccess) return r;
        return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    };
    const void* dyn[] = {(const void*)k_stage_a<float>,    (const void*)k_stage_a<double>,
                         (const void*)k_mid<float>,        (const void*)k_mid<double>,
                         (const void*)k_final<float>,      (const void*)k_final<double>,
                         (const void*)k_acorr_fft<double2>, (const void*)k_acorr_fft<dcplx>,
                         (const void*)k_spec_df,           (const void*)k_select2d_lag<1>,
                         (const void*)k_select2d_lag<2>,   (const void*)k_select2d_lag<4>,
                         (const void*)k_select2d,          (const void*)k_fused2d<float, 2>,
                         (const void*)k_fused2d<float, 4>, (const void*)k_fused2d<double, 2>};
    for (const void* f : dyn)
        if ((e = raise(f)) != cudaSuccess) return e;
    const void* clu[] = {(const void*)k_select2d, (const void*)k_fused2d<float, 2>, (const void*)k_fused2d<float, 4>,
                         (const void*)k_fused2d<double, 2>};
    for (const void* f : clu)
        if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) return e;
    return cudaSuccess;
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
