// kdefft_lscv_noalloc: LSCV value and gradient for one bandwidth matrix from
// caller-held grid counts, with no memory allocation of any kind.
//
// Why it exists: some callers cannot allocate device memory at the time they
// need an objective value -- code running under a fixed memory budget that was
// reserved up front, code called from inside another framework's allocator or
// callback, or real-time loops where a cudaMalloc (an implicit device
// synchronisation and a possible failure) is not acceptable.  The regular
// entry points allocate their work buffers on first use; this one uses a
// fixed scratch area that lives in the library image instead.
//
// Scratch: the file-scope array g_noalloc_scratch below (KDEFFT_NOALLOC_SCRATCH_BYTES,
// 32 MiB).  Every GPU that loads the library holds it until the process
// exits.  Host code cannot use the array's name as a device address (in host
// code it names a host-side stand-in), so the first call on each device takes
// the real address with cudaGetSymbolAddress while that device is current and
// caches it; make that first call before any stream capture.  All calls share
// the one array and it keeps the previous call's contents: everything that has
// to start at zero is written by the kernels themselves before it is read.
// Calls whose work overlaps on the GPU (different streams, or threads that do
// not order their streams) race on the array; order them on one stream.
//
// The work is the same as kdefft_lscv's for one bandwidth: the count spectrum
// |F(c_zp)|^2, the kernel grids T_H (Eq. 11) and the heat-equation gradient
// kernels generated inside the first FFT pass, the pruned FFT passes and the
// Parseval multiply-and-reduce; an epilogue kernel adds 2 n^-1 K_H(0)
// (Eq. 10) and its gradient and writes the caller's output.
#include <mutex>

#include <cmath>
#include <cstring>

#include "engine.cuh"
#include "kdefft.h"

namespace kdefft {

constexpr size_t kNoAllocBytes = KDEFFT_NOALLOC_SCRATCH_BYTES;
constexpr int kNaMaxItems = 8;
constexpr int kNaMaxTiles = 16384;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

std::mutex g_na_mutex;
constexpr int kNaMaxDevices = 64;
unsigned char* g_na_ptr[kNaMaxDevices] = {nullptr};

// host-side staging without heap use (guarded by g_na_mutex)
Item<float> h_items[kNaMaxItems];
Tile h_tiles[kNaMaxTiles];
float2 h_tw[MAXD * MAXP];
HEnt h_htab[HMAX * 4];

// failures are reported by the return code alone (no message buffer)
int na_fail(int code, const char* msg) {
    (void)msg;
    return code;
}

// ---- small FP64 algebra (row stride 4) -----------------------------------
bool chol4(const double* A, int d, double* L) {
    for (int i = 0; i < 16; ++i) L[i] = 0.0;
    for (int j = 0; j < d; ++j) {
        double s = A[j * 4 + j];
        for (int k = 0; k < j; ++k) s -= L[j * 4 + k] * L[j * 4 + k];
        if (!(s > 0.0) || !std::isfinite(s)) return false;
        L[j * 4 + j] = std::sqrt(s);
        for (int i = j + 1; i < d; ++i) {
            double t = A[i * 4 + j];
            for (int k = 0; k < j; ++k) t -= L[i * 4 + k] * L[j * 4 + k];
            L[i * 4 + j] = t / L[j * 4 + j];
        }
    }
    return true;
}

bool inv_det4(const double* A, int d, double* inv, double* det) {
    double L[16];
    if (!chol4(A, d, L)) return false;
    *det = 1.0;
    for (int i = 0; i < d; ++i) *det *= L[i * 4 + i] * L[i * 4 + i];
    for (int c = 0; c < d; ++c) {
        double y[4], x[4];
        for (int i = 0; i < d; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i * 4 + k] * y[k];
            y[i] = s / L[i * 4 + i];
        }
        for (int i = d - 1; i >= 0; --i) {
            double s = y[i];
            for (int k = i + 1; k < d; ++k) s -= L[k * 4 + i] * x[k];
            x[i] = s / L[i * 4 + i];
        }
        for (int i = 0; i < d; ++i) inv[i * 4 + c] = x[i];
    }
    return true;
}

double lam_max4(const double* S, int d) {
    double A[16];
    std::memcpy(A, S, sizeof(A));
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = i + 1; j < d; ++j) off += A[i * 4 + j] * A[i * 4 + j];
        if (off < 1e-300) break;
        for (int p = 0; p < d; ++p)
            for (int q = p + 1; q < d; ++q) {
                if (A[p * 4 + q] == 0.0) continue;
                const double th = (A[q * 4 + q] - A[p * 4 + p]) / (2.0 * A[p * 4 + q]);
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < d; ++k) {
                    const double a = A[k * 4 + p], b = A[k * 4 + q];
                    A[k * 4 + p] = c * a - s * b;
                    A[k * 4 + q] = s * a + c * b;
                }
                for (int k = 0; k < d; ++k) {
                    const double a = A[p * 4 + k], b = A[q * 4 + k];
                    A[p * 4 + k] = c * a - s * b;
                    A[q * 4 + k] = s * a + c * b;
                }
            }
    }
    double m = A[0];
    for (int i = 1; i < d; ++i) m = std::fmax(m, A[i * 4 + i]);
    return m;
}

bool smooth(long long x) {
    if (x < 1) return false;
    for (int p : {2, 3, 5})
        while (x % p == 0) x /= p;
    return x == 1;
}

bool radix(int P, AxisPlan& ap) {
    if (P < 2 || P > MAXP) return false;
    // at most 7 stages for P <= 4096 (3^7 = 2187); the bound only keeps
    // every write visibly inside the stage array
    int x = P, n = 0;
    while (x % 8 == 0 && n < MAXST) { ap.radix[n++] = 8; x /= 8; }
    if (x % 4 == 0 && n < MAXST) { ap.radix[n++] = 4; x /= 4; }
    if (x % 2 == 0 && n < MAXST) { ap.radix[n++] = 2; x /= 2; }
    while (x % 5 == 0 && n < MAXST) { ap.radix[n++] = 5; x /= 5; }
    while (x % 3 == 0 && n < MAXST) { ap.radix[n++] = 3; x /= 3; }
    if (x != 1) return false;
    ap.P = P;
    ap.nst = n;
    return true;
}

// ---- Hermite recurrence table (graded order, alpha_0 descending first) ---
const int kRmaxD[5] = {0, 8, 8, 8, 6};

long long comp(int m, int r) {   // compositions of m into r >= 1 parts: C(m + r - 1, r - 1)
    long long c = 1;
    for (int i = 1; i <= r - 1; ++i) c = c * (m + i) / i;
    return c;
}

int rank_of(int d, const int* a) {
    int o = 0;
    for (int k = 0; k < d; ++k) o += a[k];
    long long r = 0;
    for (int q = 0; q < o; ++q) r += comp(q, d);   // all lower orders
    int left = o;
    for (int k = 0; k < d - 1; ++k) {
        for (int v = left; v > a[k]; --v) r += comp(left - v, d - k - 1);
        left -= a[k];
    }
    return (int)r;
}

// enumerate order o in the graded order: calls f(alpha) in sequence
template <typename F>
void each_of_order(int d, int o, F f) {
    int a[MAXD] = {0};
    // odometer over (a_0 .. a_{d-2}) descending, a_{d-1} = remainder
    a[0] = o;
    for (;;) {
        int used = 0;
        for (int k = 0; k < d - 1; ++k) used += a[k];
        a[d - 1] = o - used;
        if (a[d - 1] >= 0) f(a);
        // next: decrement the last position (< d-1) that can move, refill the rest
        int k = d - 2;
        for (; k >= 0; --k) {
            if (a[k] > 0) break;
        }
        if (k < 0) return;
        a[k]--;
        int pre = 0;
        for (int m = 0; m <= k; ++m) pre += a[m];
        if (k + 1 <= d - 2) {
            a[k + 1] = o - pre;
            for (int m = k + 2; m <= d - 2; ++m) a[m] = 0;
        }
    }
}

int build_table(HEnt* tab, int* offs) {
    int n = 0;
    offs[0] = 0;
    for (int d = 1; d <= 4; ++d) {
        for (int o = 0; o <= kRmaxD[d]; ++o) {
            each_of_order(d, o, [&](const int* al) {
                HEnt e{};
                if (o > 0) {
                    int piv = 0;
                    while (al[piv] == 0) ++piv;
                    int beta[MAXD] = {0};
                    for (int k = 0; k < d; ++k) beta[k] = al[k];
                    beta[piv] -= 1;
                    e.piv = (uint8_t)piv;
                    e.par = (uint16_t)rank_of(d, beta);
                    for (int j = 0; j < d; ++j)
                        if (beta[j] > 0) {
                            int g[MAXD];
                            for (int k = 0; k < d; ++k) g[k] = beta[k];
                            g[j] -= 1;
                            e.rj[e.nred] = (uint8_t)j;
                            e.rc[e.nred] = (uint8_t)beta[j];
                            e.ridx[e.nred] = (uint16_t)rank_of(d, g);
                            e.nred++;
                        }
                }
                tab[n++] = e;
            });
        }
        offs[d] = n;
    }
    return n;
}

// ---- epilogue: objective assembly into the caller's buffer ----------------
__global__ void k_na_epilogue(const double* __restrict__ raw, int ngrid, double c0, const double* __restrict__ cg,
                              int d, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    // raw holds (re, im) per item; grid g sits at raw[g] (items pack grids in order)
    out[0] = raw[0] + c0;
    int g = 1;
    for (int a = 0; a < d; ++a)
        for (int b = a; b < d; ++b) {
            const double v = raw[g] + cg[a * 4 + b];
            out[1 + a * d + b] = v;
            out[1 + b * d + a] = v;
            ++g;
        }
    (void)ngrid;
}

// one-time set-up for the current device: the scratch address, the
// Hermite tables in constant memory and the kernels' shared-memory limits
// (raised once, so that no call sets them)
int na_setup(int dev, unsigned char** base) {
    if (dev < 0 || dev >= kNaMaxDevices) return na_fail(KDEFFT_ERR_UNSUPPORTED, "device index too large");
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return na_fail(KDEFFT_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed");
        int offs[5];
        const int n = build_table(h_htab, offs);
        if (upload_hermite_tables(h_htab, offs, n) != cudaSuccess)
            return na_fail(KDEFFT_ERR_CUDA, "Hermite table upload failed");
        if (prepare_kernels() != cudaSuccess) return na_fail(KDEFFT_ERR_CUDA, "kernel attributes failed");
        g_na_ptr[dev] = (unsigned char*)p;
    }
    *base = g_na_ptr[dev];
    return KDEFFT_OK;
}

}  // namespace
}  // namespace kdefft

using namespace kdefft;

extern "C" int kdefft_lscv_noalloc(int d, const int64_t* M, const double* delta, int64_t n, const float* counts,
                                   const double* H, double tau, void* stream, double* out) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (d < 1 || d > 3 || !M || !delta || !counts || !H || !out || n < 2 || !(tau > 0.0))
        return na_fail(KDEFFT_ERR_ARG, "bad argument (d must be 1..3, n >= 2, tau > 0, non-null arrays)");
    cudaStream_t st = (cudaStream_t)stream;
    {
        // The small tables go up from host staging that the next call
        // overwrites; a captured copy would replay whatever a later call left
        // there.  So the call does nothing while its stream is being captured.
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
            return na_fail(KDEFFT_ERR_UNSUPPORTED, "the stream is being captured");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return na_fail(KDEFFT_ERR_CUDA, "no current CUDA device");
    {
        // both buffers must be device memory of the current device: a peer
        // device's buffer would be read without peer access
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, out) != cudaSuccess || a.type != cudaMemoryTypeDevice || a.device != dev) {
            cudaGetLastError();
            return na_fail(KDEFFT_ERR_ARG, "out must be device memory of the current device");
        }
        if (cudaPointerGetAttributes(&a, counts) != cudaSuccess || a.type != cudaMemoryTypeDevice ||
            a.device != dev) {
            cudaGetLastError();
            return na_fail(KDEFFT_ERR_ARG, "counts must be device memory of the current device");
        }
    }
    unsigned char* base = nullptr;
    int r = na_setup(dev, &base);
    if (r != KDEFFT_OK) return r;

    // ---- bandwidth algebra, support L (Eq. 26) and minimal padding
    double Hm[16] = {0}, H2[16] = {0}, inv[16], det, inv2[16], det2;
    double mx = 0.0;
    for (int i = 0; i < d * d; ++i) mx = std::fmax(mx, std::fabs(H[i]));
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            if (std::fabs(H[i * d + j] - H[j * d + i]) > 1e-12 * mx) return na_fail(KDEFFT_ERR_ARG, "H not symmetric");
            Hm[i * 4 + j] = 0.5 * (H[i * d + j] + H[j * d + i]);
            H2[i * 4 + j] = 2.0 * Hm[i * 4 + j];
        }
    if (!inv_det4(Hm, d, inv, &det) || !inv_det4(H2, d, inv2, &det2))
        return na_fail(KDEFFT_ERR_NOT_SPD, "H is not positive definite");
    const double lam = lam_max4(Hm, d);
    int L[MAXD] = {0}, P[MAXD] = {0};
    long long ptot = 1;
    for (int k = 0; k < d; ++k) {
        if (M[k] < 2 || M[k] > MAXP) return na_fail(KDEFFT_ERR_UNSUPPORTED, "M_k out of range");
        double c = std::ceil(tau * std::sqrt(std::fabs(lam)) / delta[k]);
        if (!(c <= (double)(M[k] - 1))) c = (double)(M[k] - 1);
        if (c < 1.0) c = 1.0;
        L[k] = (int)c;
        long long p = M[k] + L[k];
        while (!smooth(p)) ++p;
        if (p > MAXP) return na_fail(KDEFFT_ERR_UNSUPPORTED, "padded size above 4096");
        P[k] = (int)p;
        ptot *= p;
    }

    // ---- twiddles for the distinct P (staged in scratch)
    int tw_off[MAXD];
    int ntw = 0;
    for (int k = 0; k < d; ++k) {
        int found = -1;
        for (int m = 0; m < k; ++m)
            if (P[m] == P[k]) found = tw_off[m];
        if (found >= 0) {
            tw_off[k] = found;
            continue;
        }
        tw_off[k] = ntw;
        for (int t = 0; t < P[k]; ++t) {
            const long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)t / (long double)P[k];
            h_tw[ntw + t] = make_float2((float)(double)cosl(ang), (float)(double)sinl(ang));
        }
        ntw += P[k];
    }

    // ---- items: 0 = counts spectrum; then the packed LSCV grid pairs
    const int ngrid = 1 + d * (d + 1) / 2;
    const int nkitems = (ngrid + 1) / 2;
    const int nitems = 1 + nkitems;
    long long spec = (long long)(P[d - 1] / 2 + 1);
    for (int k = 0; k < d - 1; ++k) spec *= P[k];
    for (int i = 0; i < nitems; ++i) std::memset(&h_items[i], 0, sizeof(Item<float>));
    for (int i = 0; i < nitems; ++i) {
        Item<float>& it = h_items[i];
        it.d = d;
        it.kind = (i == 0) ? 1 : 0;
        for (int k = 0; k < d; ++k) {
            if (!radix(P[k], it.ax[k])) return na_fail(KDEFFT_ERR_UNSUPPORTED, "no radix plan");
            it.ax[k].tw_off = tw_off[k];
            it.S[k] = (i == 0) ? (int)M[k] : 2 * L[k] + 1;
            it.off[k] = (i == 0) ? 0 : L[k];
            it.delta[k] = delta[k];
        }
        it.scale = 1.0 / ((double)n * (double)n * (double)ptot);
    }
    // grid list: T = phi_2H - 2 phi_H; G_ab = s (d_a d_b phi_2H - d_a d_b phi_H)
    for (int g = 0; g < ngrid; ++g) {
        Item<float>& it = h_items[1 + g / 2];
        const int h = g & 1;
        it.nsig = 2;
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                it.lam[0][a * MAXD + b] = inv2[a * 4 + b];
                it.lam[1][a * MAXD + b] = inv[a * 4 + b];
            }
        it.nrm[0] = std::pow(2.0 * M_PI, -0.5 * d) / std::sqrt(det2);
        it.nrm[1] = std::pow(2.0 * M_PI, -0.5 * d) / std::sqrt(det);
        int al[MAXD] = {0};
        float w0 = 1.0f, w1 = -2.0f;
        if (g > 0) {
            int gi = 1, A = 0, B = 0;
            for (int a = 0; a < d; ++a)
                for (int b = a; b < d; ++b) {
                    if (gi == g) { A = a; B = b; }
                    ++gi;
                }
            al[A] += 1;
            al[B] += 1;
            const float s = (A == B) ? 1.0f : 2.0f;
            w0 = s;
            w1 = -s;
            it.R = 2;
        }
        it.nterm[h] = 2;
        it.tsig[h][0] = 0;
        it.tsig[h][1] = 1;
        it.the[h][0] = (short)rank_of(d, al);
        it.the[h][1] = (short)rank_of(d, al);
        it.tw8[h][0] = w0;   // order 0 or 2: sign (-1)^{|alpha|} = +1
        it.tw8[h][1] = w1;
    }

    // ---- scratch layout and tiles
    const int cap = 6144;
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    const size_t o_tw = off;
    off = align(off + sizeof(float2) * ntw);
    const size_t o_spec = off;
    off = align(off + sizeof(float) * spec);
    const size_t o_items = off;
    off = align(off + sizeof(Item<float>) * nitems);
    const size_t o_raw = off;
    off = align(off + sizeof(double) * 2 * nitems);
    // per pipeline: stage scratch + tiles + partials (counts then kernels reuse it)
    long long scr_elems = 0;
    int nt = 0;
    int tA[2], tM[2], tF[2], nA[2], nM[2], nF[2], capA[2], capM[2], capF[2];
    for (int pass = 0; pass < 2; ++pass) {
        const int i0 = (pass == 0) ? 0 : 1, i1 = (pass == 0) ? 1 : nitems;
        long long sc = 0;
        // stage A
        tA[pass] = nt;
        capA[pass] = 0;
        for (int i = i0; i < i1; ++i) {
            Item<float>& it = h_items[i];
            const int Pl = P[d - 1], Ql = Pl / 2 + 1;
            long long lines = 1;
            for (int k = 0; k < d - 1; ++k) lines *= it.S[k];
            const int nl = (int)std::max<long long>(1, std::min<long long>(cap / Pl, lines));
            for (long long l0 = 0; l0 < lines; l0 += nl) {
                if (nt >= kNaMaxTiles) return na_fail(KDEFFT_ERR_UNSUPPORTED, "too many tiles for the no-alloc path");
                const int cnt = (int)std::min<long long>(nl, lines - l0);
                h_tiles[nt++] = Tile{i, (int)l0, 0, cnt};
                capA[pass] = std::max(capA[pass], cnt * Pl);
            }
            long long sz0 = (d >= 2) ? (long long)Ql * lines : 0, sz1 = 0, Wo = Ql;
            int wsel = 0;
            for (int k = d - 2; k >= 1; --k) {
                long long O = 1;
                for (int m = 0; m < k; ++m) O *= it.S[m];
                Wo *= P[k];
                wsel ^= 1;
                (wsel ? sz1 : sz0) = std::max(wsel ? sz1 : sz0, Wo * O);
            }
            it.scr[0] = sc;
            it.scr[1] = sc + sz0;
            sc += sz0 + sz1;
        }
        nA[pass] = nt - tA[pass];
        // mid pass (d = 3: axis 1)
        tM[pass] = nt;
        capM[pass] = 0;
        if (d == 3) {
            for (int i = i0; i < i1; ++i) {
                Item<float>& it = h_items[i];
                const long long Wo = (long long)(P[2] / 2 + 1);
                const long long O = it.S[0];
                const int nl = (int)std::max<long long>(1, std::min<long long>(cap / P[1], O));
                for (long long wo = 0; wo < Wo; ++wo)
                    for (long long o0 = 0; o0 < O; o0 += nl) {
                        if (nt >= kNaMaxTiles)
                            return na_fail(KDEFFT_ERR_UNSUPPORTED, "too many tiles for the no-alloc path");
                        const int cnt = (int)std::min<long long>(nl, O - o0);
                        h_tiles[nt++] = Tile{i, (int)wo, (int)o0, cnt};
                        capM[pass] = std::max(capM[pass], cnt * P[1]);
                    }
            }
        }
        nM[pass] = nt - tM[pass];
        // final pass (d >= 2)
        tF[pass] = nt;
        capF[pass] = 0;
        if (d >= 2) {
            for (int i = i0; i < i1; ++i) {
                Item<float>& it = h_items[i];
                long long Wo = P[d - 1] / 2 + 1;
                for (int k = 1; k <= d - 2; ++k) Wo *= P[k];
                const int nl = (int)std::max<long long>(1, std::min<long long>(cap / P[0], Wo));
                it.tileF0 = nt - tF[pass];
                int cnt_tiles = 0;
                for (long long q0 = 0; q0 < Wo; q0 += nl) {
                    if (nt >= kNaMaxTiles) return na_fail(KDEFFT_ERR_UNSUPPORTED, "too many tiles for the no-alloc path");
                    const int cnt = (int)std::min<long long>(nl, Wo - q0);
                    h_tiles[nt++] = Tile{i, (int)q0, 0, cnt};
                    capF[pass] = std::max(capF[pass], cnt * P[0]);
                    ++cnt_tiles;
                }
                it.ntileF = cnt_tiles;
            }
        } else {
            for (int i = i0; i < i1; ++i) {
                h_items[i].tileF0 = i - i0;
                h_items[i].ntileF = 1;
            }
        }
        nF[pass] = nt - tF[pass];
        scr_elems = std::max(scr_elems, sc);
    }
    const size_t o_tiles = off;
    off = align(off + sizeof(Tile) * nt);
    const size_t o_part = off;
    off = align(off + sizeof(double) * 2 * (size_t)std::max(nF[0], std::max(nF[1], nitems)));
    const size_t o_scr = off;
    off = align(off + sizeof(float2) * (size_t)scr_elems);
    const size_t o_cg = off;
    off = align(off + sizeof(double) * 16);
    if (off > kNoAllocBytes) return na_fail(KDEFFT_ERR_UNSUPPORTED, "problem exceeds the 32 MiB no-alloc scratch");

    float2* d_tw = (float2*)(base + o_tw);
    float* d_spec = (float*)(base + o_spec);
    Item<float>* d_items = (Item<float>*)(base + o_items);
    double* d_raw = (double*)(base + o_raw);
    Tile* d_tiles = (Tile*)(base + o_tiles);
    double* d_part = (double*)(base + o_part);
    float2* d_scr = (float2*)(base + o_scr);
    double* d_cg = (double*)(base + o_cg);
    h_items[0].counts = counts;
    h_items[0].spec_out = d_spec;
    for (int i = 1; i < nitems; ++i) h_items[i].spec = d_spec;

    // gradient constants of 2 n^-1 K_H(0): -n^-1 K_H(0) H^{-1}, tied off-diagonals doubled
    const double k0 = std::pow(2.0 * M_PI, -0.5 * d) / std::sqrt(det);
    double cg[16] = {0};
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) cg[a * 4 + b] = (2.0 / (double)n) * ((a == b) ? 1.0 : 2.0) * (-0.5 * k0 * inv[a * 4 + b]);

#define NA_CU(x)                                                                  \
    do {                                                                          \
        if ((x) != cudaSuccess) return na_fail(KDEFFT_ERR_CUDA, #x " failed");    \
    } while (0)
    NA_CU(cudaMemcpyAsync(d_tw, h_tw, sizeof(float2) * ntw, cudaMemcpyHostToDevice, st));
    NA_CU(cudaMemcpyAsync(d_items, h_items, sizeof(Item<float>) * nitems, cudaMemcpyHostToDevice, st));
    NA_CU(cudaMemcpyAsync(d_tiles, h_tiles, sizeof(Tile) * nt, cudaMemcpyHostToDevice, st));
    NA_CU(cudaMemcpyAsync(d_cg, cg, sizeof(cg), cudaMemcpyHostToDevice, st));
    int nsm = 1;
    NA_CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    auto grid = [&](int ntiles) { return std::max(1, std::min(ntiles, nsm * 4)); };
    int pmax = 0;
    for (int k = 0; k < d; ++k) pmax = std::max(pmax, P[k]);
    for (int pass = 0; pass < 2; ++pass) {
        if (nA[pass] > 0)
            NA_CU(launch_stage_a<float>(d_items, d_tiles + tA[pass], nA[pass], pmax, capA[pass], d_scr, d_tw,
                                        d_part, grid(nA[pass]), st));
        if (nM[pass] > 0)
            NA_CU(launch_mid<float>(d_items, d_tiles + tM[pass], nM[pass], 1, pmax, capM[pass], d_scr, d_tw,
                                    grid(nM[pass]), st));
        if (nF[pass] > 0)
            NA_CU(launch_final<float>(d_items, d_tiles + tF[pass], nF[pass], pmax, capF[pass], d_scr, d_tw, d_part,
                                      grid(nF[pass]), st));
    }
    // kernel items are items 1..; reduce them into raw[2 * (i - 1) + {0, 1}]
    NA_CU(launch_reduce<float>(d_items + 1, nkitems, d_part, d_raw, st));
    k_na_epilogue<<<1, 32, 0, st>>>(d_raw, ngrid, 2.0 * k0 / (double)n, d_cg, d, out);
    NA_CU(cudaGetLastError());
#undef NA_CU
    return KDEFFT_OK;
}
