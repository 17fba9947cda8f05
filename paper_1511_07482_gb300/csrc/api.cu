// Host side of the library and the C ABI declared in include/kdefft.h.
//
// Responsibilities (the device does all per-sample and per-grid-point work):
//   - FP64 bandwidth algebra: symmetrisation, Cholesky (SPD check), inverse,
//     determinant, largest eigenvalue (Jacobi) -> L_k (Eq. 26), P_k (Eqs. 21,
//     27 or the minimal no-alias length);
//   - kernel descriptions: which Gaussian partials, covariances and weights
//     make each lag kernel (T_H of Eq. 11, heat-equation gradient kernels,
//     the SCV kernel, psi_r partials, eta_{0,2});
//   - work lists: pairs of real kernels packed into one complex transform,
//     tiles of each pass, scratch offsets; one launch sequence per batch;
//   - objective assembly in FP64 (adding 2 n^-1 K_H(0) etc.);
//   - the quasi-Newton bandwidth optimiser of kdefft_select_H.
#include <algorithm>
#include <array>
#include <atomic>
#include <functional>
#include <thread>
#include <set>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "engine.cuh"
#include "kdefft.h"

using namespace kdefft;

// ============================================================ errors
// Run fn(i0, i1) over [0, n) split into contiguous ranges: inline below two
// grains, else on up to four host threads (the caller's among them).  The
// grains keep work of a few hundred microseconds on one thread: starting the
// threads costs about as much (measured: the 3-D psi_4 batch got slower with
// its 2048 lag items split four ways).  Each
// range's results go to entries of their own, so the outcome does not depend
// on the split; fn reports failures through shared flags, never through
// fail() (whose message is per thread).
template <typename F>
static void host_parallel_for(size_t n, size_t grain, F&& fn) {
    if (n < 2 * std::max<size_t>(grain, 1)) {
        if (n) fn((size_t)0, n);
        return;
    }
    // (the core count is read once: the query reads a system file)
    static const unsigned hc = std::max(1u, std::thread::hardware_concurrency());
    const size_t parts = std::min<size_t>({(size_t)4, (size_t)hc, n / std::max<size_t>(grain, 1)});
    if (parts < 2) {
        fn((size_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(parts - 1);
    const size_t per = (n + parts - 1) / parts;
    for (size_t k = 1; k < parts; ++k) {
        const size_t a = k * per, b = std::min(n, a + per);
        if (a < b) th.emplace_back([&fn, a, b] { fn(a, b); });
    }
    fn((size_t)0, std::min(n, per));
    for (std::thread& t : th) t.join();
}

static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define KCU(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail(KDEFFT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define KCHK(expr)              \
    do {                        \
        int r_ = (expr);        \
        if (r_ != KDEFFT_OK) return r_; \
    } while (0)

// ============================================================ buffers
// Device blocks of datasets return, when a dataset is destroyed or a buffer
// grows, to their context's cache and are reused by later datasets.  All of
// a context's work runs in the order of its stream, so a block taken from
// the cache is only touched after the work that used it before.  A dataset
// per step then costs no cudaMalloc and no cudaFree (each cudaFree
// synchronises the device).
struct BlockCache {
    std::multimap<size_t, void*> blocks;   // capacity -> free block
    size_t bytes = 0;                      // held in free blocks
    size_t limit = (size_t)16 << 30;       // free blocks beyond this are returned to CUDA
    int64_t hits = 0, misses = 0;
    // a free block of at least `want` bytes and at most twice that, or null
    void* take(size_t want, size_t& cap) {
        auto it = blocks.lower_bound(want);
        if (it == blocks.end() || it->first > 2 * want) return nullptr;
        cap = it->first;
        void* q = it->second;
        blocks.erase(it);
        bytes -= cap;
        ++hits;
        return q;
    }
    void give(void* q, size_t cap) {
        blocks.emplace(cap, q);
        bytes += cap;
        while (bytes > limit && !blocks.empty()) {   // the largest go first
            auto it = std::prev(blocks.end());
            cudaFree(it->second);
            bytes -= it->first;
            blocks.erase(it);
        }
    }
    void trim() {
        for (auto& kv : blocks) cudaFree(kv.second);
        blocks.clear();
        bytes = 0;
    }
};

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    bool owner = true;   // false: a view into memory another buffer owns
    BlockCache* cache = nullptr;   // where owned blocks come from and go back to (null: cudaMalloc / cudaFree)
    int64_t* gen = nullptr;        // bumped whenever the block changes (graphs that captured it go stale)
    DevBuf() = default;
    explicit DevBuf(BlockCache* bc) : cache(bc) {}
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void view(void* q, size_t bytes) {
        release();
        p = q;
        cap = bytes;
        owner = false;
    }
    int ensure(size_t bytes) {
        if (bytes <= cap) return KDEFFT_OK;
        release();
        size_t want = std::max(bytes, (size_t)4096);
        if (cache) {
            size_t got = 0;
            if (void* q = cache->take(want, got)) {
                p = q;
                cap = got;
                if (gen) ++*gen;
                return KDEFFT_OK;
            }
            ++cache->misses;
        }
        want = want + want / 4;
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, want);
        if (e != cudaSuccess && cache && cache->bytes) {   // give the cached blocks back and try once more
            cudaGetLastError();
            cache->trim();
            q = nullptr;
            e = cudaMalloc(&q, want);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(KDEFFT_ERR_ALLOC, "device allocation of " + std::to_string(want) + " bytes failed");
        }
        p = q;
        cap = want;
        if (gen) ++*gen;
        return KDEFFT_OK;
    }
    void release() {
        if (p && owner) {
            if (cache)
                cache->give(p, cap);
            else
                cudaFree(p);
            if (gen) ++*gen;
        }
        p = nullptr;
        cap = 0;
        owner = true;
    }
};

struct HostBuf {
    void* p = nullptr;
    size_t cap = 0;
    int64_t* gen = nullptr;   // as DevBuf::gen
    HostBuf() = default;
    HostBuf(const HostBuf&) = delete;
    HostBuf& operator=(const HostBuf&) = delete;
    ~HostBuf() { release(); }
    int ensure(size_t bytes) {
        if (bytes <= cap) return KDEFFT_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        size_t want = std::max(bytes, (size_t)4096);
        want = want + want / 4;
        if (gen) ++*gen;
        if (cudaMallocHost(&p, want) != cudaSuccess) {
            p = nullptr;
            return fail(KDEFFT_ERR_ALLOC, "pinned host allocation failed");
        }
        cap = want;
        return KDEFFT_OK;
    }
    void release() {
        if (p) {
            cudaFreeHost(p);
            if (gen) ++*gen;
        }
        p = nullptr;
        cap = 0;
    }
};

static bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ============================================================ small FP64 matrices (row stride 4)
struct Mat {
    int d = 0;
    double a[16] = {0};
    double& operator()(int i, int j) { return a[i * 4 + j]; }
    double operator()(int i, int j) const { return a[i * 4 + j]; }
};

static Mat mat_from(const double* H, int d) {
    Mat m;
    m.d = d;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) m(i, j) = H[i * d + j];
    return m;
}

static Mat lin(double a, const Mat& A, double b, const Mat& B) {
    Mat m;
    m.d = A.d;
    for (int i = 0; i < A.d; ++i)
        for (int j = 0; j < A.d; ++j) m(i, j) = a * A(i, j) + b * B(i, j);
    return m;
}

static Mat scaled(double a, const Mat& A) { return lin(a, A, 0.0, A); }

// symmetric check (relative 1e-12) and symmetrisation
static int sym_check(const double* H, int d, Mat& out, const char* name) {
    double mx = 0.0;
    for (int i = 0; i < d * d; ++i) {
        if (!std::isfinite(H[i])) return fail(KDEFFT_ERR_ARG, std::string(name) + " has a non-finite entry");
        mx = std::max(mx, std::fabs(H[i]));
    }
    out = mat_from(H, d);
    for (int i = 0; i < d; ++i)
        for (int j = i + 1; j < d; ++j) {
            if (std::fabs(out(i, j) - out(j, i)) > 1e-12 * mx)
                return fail(KDEFFT_ERR_ARG, std::string(name) + " is not symmetric");
            const double s = 0.5 * (out(i, j) + out(j, i));
            out(i, j) = out(j, i) = s;
        }
    return KDEFFT_OK;
}

static bool cholesky(const Mat& A, Mat& L) {
    const int d = A.d;
    L = Mat();
    L.d = d;
    for (int j = 0; j < d; ++j) {
        double s = A(j, j);
        for (int k = 0; k < j; ++k) s -= L(j, k) * L(j, k);
        if (!(s > 0.0) || !std::isfinite(s)) return false;
        L(j, j) = std::sqrt(s);
        for (int i = j + 1; i < d; ++i) {
            double t = A(i, j);
            for (int k = 0; k < j; ++k) t -= L(i, k) * L(j, k);
            L(i, j) = t / L(j, j);
        }
    }
    return true;
}

// inverse and determinant of an SPD matrix from its Cholesky factor
static bool spd_inv_det(const Mat& A, Mat& inv, double& det) {
    Mat L;
    if (!cholesky(A, L)) return false;
    const int d = A.d;
    det = 1.0;
    for (int i = 0; i < d; ++i) det *= L(i, i) * L(i, i);
    // solve A x = e_c for each column
    inv = Mat();
    inv.d = d;
    for (int c = 0; c < d; ++c) {
        double y[4], x[4];
        for (int i = 0; i < d; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L(i, k) * y[k];
            y[i] = s / L(i, i);
        }
        for (int i = d - 1; i >= 0; --i) {
            double s = y[i];
            for (int k = i + 1; k < d; ++k) s -= L(k, i) * x[k];
            x[i] = s / L(i, i);
        }
        for (int i = 0; i < d; ++i) inv(i, c) = x[i];
    }
    for (int i = 0; i < d; ++i)
        for (int j = i + 1; j < d; ++j) inv(i, j) = inv(j, i) = 0.5 * (inv(i, j) + inv(j, i));
    return true;
}

// largest eigenvalue of a symmetric matrix, cyclic Jacobi rotations, until
// the off-diagonal mass is below 1e-32 of the squared Frobenius norm: by
// Weyl's bound every diagonal entry is then within about 1.4e-16 |S|_F of an
// eigenvalue (machine precision); 3-4 sweeps for d = 3 instead of the ~10
// that driving it to zero took (a quarter of the host time of a batch of
// bandwidths)
static double lambda_max(const Mat& S) {
    const int d = S.d;
    Mat A = S;
    double fro = 0.0;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) fro += A(i, j) * A(i, j);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = i + 1; j < d; ++j) off += A(i, j) * A(i, j);
        if (!(off > 1e-32 * fro)) break;
        for (int p = 0; p < d; ++p)
            for (int q = p + 1; q < d; ++q) {
                if (A(p, q) == 0.0) continue;
                const double theta = (A(q, q) - A(p, p)) / (2.0 * A(p, q));
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < d; ++k) {
                    const double akp = A(k, p), akq = A(k, q);
                    A(k, p) = c * akp - s * akq;
                    A(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < d; ++k) {
                    const double apk = A(p, k), aqk = A(q, k);
                    A(p, k) = c * apk - s * aqk;
                    A(q, k) = s * apk + c * aqk;
                }
            }
    }
    double m = A(0, 0);
    for (int i = 1; i < d; ++i) m = std::max(m, A(i, i));
    return m;
}

// ============================================================ Hermite recurrence tables
static const int kRmax[5] = {0, 8, 8, 8, 6};

struct MultiIndex {
    int a[MAXD];
};

// graded enumeration: order 0, 1, ..., R; within an order alpha_0 descending,
// then alpha_1 descending, ...
static void enumerate(int d, int R, std::vector<MultiIndex>& out) {
    out.clear();
    for (int o = 0; o <= R; ++o) {
        std::vector<MultiIndex> lvl;
        MultiIndex m{};
        std::function<void(int, int)> rec = [&](int k, int left) {
            if (k == d - 1) {
                m.a[k] = left;
                lvl.push_back(m);
                return;
            }
            for (int v = left; v >= 0; --v) {
                m.a[k] = v;
                rec(k + 1, left - v);
            }
        };
        rec(0, o);
        out.insert(out.end(), lvl.begin(), lvl.end());
    }
}

struct HermiteIndex {
    std::vector<MultiIndex> list[5];
    std::vector<int> code[5];   // alpha as base-9 digits -> position in the graded order
    static int key(int d, const int* a) {
        int k = 0;
        for (int i = 0; i < d; ++i) k = k * 9 + a[i];
        return k;
    }
    int idx(int d, const int* a) const {
        for (int i = 0; i < d; ++i)
            if (a[i] < 0 || a[i] > 8) return -1;
        return code[d][key(d, a)];
    }
};

// built once, on first use (a function-local static: thread-safe initialisation)
static HermiteIndex& hindex() {
    static HermiteIndex h = [] {
        HermiteIndex x;
        for (int d = 1; d <= 4; ++d) {
            enumerate(d, kRmax[d], x.list[d]);
            int n = 1;
            for (int i = 0; i < d; ++i) n *= 9;
            x.code[d].assign(n, -1);
            for (size_t t = 0; t < x.list[d].size(); ++t) x.code[d][HermiteIndex::key(d, x.list[d][t].a)] = (int)t;
        }
        return x;
    }();
    return h;
}

static int upload_tables() {
    HermiteIndex& h = hindex();
    std::vector<HEnt> tab;
    int offs[5];
    offs[0] = 0;
    for (int d = 1; d <= 4; ++d) {
        for (size_t t = 0; t < h.list[d].size(); ++t) {
            HEnt e{};
            if (t > 0) {
                const MultiIndex& al = h.list[d][t];
                int piv = 0;
                while (al.a[piv] == 0) ++piv;
                int beta[MAXD] = {0};
                for (int k = 0; k < d; ++k) beta[k] = al.a[k];
                beta[piv] -= 1;
                e.piv = (uint8_t)piv;
                e.par = (uint16_t)h.idx(d, beta);
                e.nred = 0;
                for (int j = 0; j < d; ++j)
                    if (beta[j] > 0) {
                        int g[MAXD];
                        for (int k = 0; k < d; ++k) g[k] = beta[k];
                        g[j] -= 1;
                        e.rj[e.nred] = (uint8_t)j;
                        e.rc[e.nred] = (uint8_t)beta[j];
                        e.ridx[e.nred] = (uint16_t)h.idx(d, g);
                        e.nred++;
                    }
            }
            tab.push_back(e);
        }
        offs[d] = (int)tab.size();
    }
    KCU(upload_hermite_tables(tab.data(), offs, (int)tab.size()));
    return KDEFFT_OK;
}

// ============================================================ radix plans & twiddles
// Radices the device passes implement (register DFTs; composite ones as a
// compile-time mixed-radix decomposition), largest first.  FP64 lines keep
// radices <= 16 (register budget).
static const int kRadices[] = {32, 30, 27, 25, 24, 20, 18, 16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};

// fewest stages factoring P into allowed radices (cached per (P, max radix))
static bool radix_plan_uncached(int P, AxisPlan& ap, int max_radix);
static bool radix_plan(int P, AxisPlan& ap, int max_radix) {
    // shared by every context of the process, so guarded for contexts used
    // from several host threads
    static std::mutex mu;
    static std::map<std::pair<int, int>, std::pair<bool, AxisPlan>> cache;
    const auto key = std::make_pair(P, max_radix);
    std::pair<bool, AxisPlan> hit;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it == cache.end()) {
            AxisPlan a{};
            const bool ok = radix_plan_uncached(P, a, max_radix);
            it = cache.emplace(key, std::make_pair(ok, a)).first;
        }
        hit = it->second;
    }
    const int tw_off = ap.tw_off;
    ap = hit.second;
    ap.tw_off = tw_off;
    return hit.first;
}

static bool radix_plan_uncached(int P, AxisPlan& ap, int max_radix) {
    if (P < 2 || P > MAXP) return false;
    // best[p]: minimal stage count for the cofactor p (dynamic programming over divisors)
    std::map<int, std::pair<int, int>> memo;   // p -> (stages, first radix)
    std::function<int(int)> best = [&](int p) -> int {
        if (p == 1) return 0;
        auto it = memo.find(p);
        if (it != memo.end()) return it->second.first;
        int bs = 1 << 20, br = 0;
        for (int r : kRadices) {
            if (r > max_radix || p % r) continue;
            const int c = 1 + best(p / r);
            if (c < bs) {
                bs = c;
                br = r;
            }
        }
        memo[p] = {bs, br};
        return bs;
    };
    if (best(P) >= (1 << 20)) return false;
    int n = 0;
    for (int p = P; p > 1;) {
        const int r = memo[p].second;
        if (n >= MAXST) return false;
        ap.radix[n++] = (unsigned char)r;
        p /= r;
    }
    ap.P = P;
    ap.nst = n;
    return true;
}

extern "C" int kdefft_radix_plan(int P, int max_radix, int* radices, int* nstages) {
    if (!radices || !nstages) return fail(KDEFFT_ERR_ARG, "NULL argument");
    AxisPlan ap{};
    if (!radix_plan(P, ap, max_radix)) return fail(KDEFFT_ERR_UNSUPPORTED, "no radix schedule for this length");
    *nstages = ap.nst;
    for (int i = 0; i < ap.nst; ++i) radices[i] = ap.radix[i];
    return KDEFFT_OK;
}

static bool is_smooth(long long x) {
    if (x < 1) return false;
    for (int p : {2, 3, 5})
        while (x % p == 0) x /= p;
    return x == 1;
}

// smallest 2^a 3^b 5^c >= m: a table up to 8192 (built once, thread-safe
// initialisation of a function-local static; the search loop cost about half
// of the request building of a large batch of bandwidths), a search above
static long long next_smooth(long long m) {
    constexpr int kTab = 8192;
    static const std::vector<int> tab = [] {
        std::vector<int> t(kTab + 1);
        int next = kTab + 1;
        while (!is_smooth(next)) ++next;
        for (int x = kTab; x >= 1; --x) {
            if (is_smooth(x)) next = x;
            t[x] = next;
        }
        t[0] = 1;
        return t;
    }();
    if (m <= kTab) return tab[m < 0 ? 0 : m];
    while (!is_smooth(m)) ++m;
    return m;
}

// ============================================================ context & dataset
struct kdefft_ds_s;
struct ReqSet;

struct kdefft_ctx_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    int nsm = 1;
    std::map<int, int> tw_off;
    std::vector<double> tw_host;      // interleaved re, im
    DevBuf tw32, tw64, twdf;          // twiddles in FP32, FP64 and FP32 pairs
    size_t tw_dev_n = 0;              // twiddles resident on the device
    DevBuf scratch, partial, items, tiles, out;
    HostBuf h_items, h_out;
    // lag-domain results on their way to h_out, not yet read: run_lag returns
    // without waiting, and flush_reads (at the end of run()) waits once for
    // all of them
    struct PendingRead {
        ReqSet* rs;
        std::vector<std::pair<int, int>> pairs;   // grid pairs in the order of their results
        size_t off;                               // first double in h_out
    };
    std::vector<PendingRead> pend_reads;
    size_t hout_used = 0;       // doubles of h_out holding pending results
    bool staging_free = true;   // no copy out of h_items is pending on the stream
    cudaEvent_t staging_ev = nullptr;   // recorded after the last copy out of h_items
    // counters: kernel launches and host<->device bytes (always), per-kernel
    // CUDA-event times and algorithmic bytes/flops (when profiling is on)
    struct KStat {
        int64_t launches = 0;
        double ms = 0.0, bytes = 0.0, flops = 0.0;
    };
    bool prof = false;
    bool fused = true;    // d = 2: single cluster kernel per batch when it fits
    bool lag = true;      // lag-domain engine for grids whose padding has no aliasing
    int* errflag = nullptr;   // device flag: a bounded device-side wait gave up
    int max_cluster = 16;     // largest cluster the fused engine may launch
    bool device_select = true;   // d = 2 FP32 selections run as one device-resident launch
    BlockCache cache;         // freed dataset blocks for reuse (declared before the buffers it serves)
    DevBuf sel_buf;           // device tables and start states of the device-resident selection
    DevBuf binfix;            // fixed-point accumulators of FP32 linear binning (stream-ordered reuse)
    DevBuf acbuf[2];          // pass buffers of the autocorrelation (stream-ordered reuse)
    DevBuf acjobs;            // job table of the batched autocorrelation passes
    HostBuf h_acjobs;         // its pinned staging copy, free once acjobs_ev has passed
    HostBuf h_sel;            // pinned start / end table of the lag-domain device search
    HostBuf h_binres;         // pinned outside count and moment partials of a binning
    cudaEvent_t acjobs_ev = nullptr;
    bool acjobs_free = true;
    DevBuf specjobs;          // job table of the FP32-pair count-spectrum passes
    HostBuf h_specjobs;       // its pinned staging copy, free once specjobs_ev has passed
    cudaEvent_t specjobs_ev = nullptr;
    bool specjobs_free = true;
    DevBuf binjobs;           // job tables of the batched binning
    DevBuf kdebuf;            // stencil table / outputs of the grid estimate and the mixture term
    std::map<std::string, KStat> kstat;
    struct Pending {
        std::string name;
        cudaEvent_t a, b;
        double bytes, flops;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> evpool;
    int64_t launches = 0, h2d = 0, d2h = 0;
    std::vector<kdefft_ds> datasets;   // live datasets; destroyed with the context
    // CUDA graphs of repeated launch sequences, keyed by launch signature
    bool graphs = true;
    cudaStream_t cap_stream = nullptr;   // capture stream, created on first use
    // second stream for launches that run beside the main stream's (the
    // FP64 lag batch of a run beside its FP32 one), forked and joined by the
    // two events; created on first use
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    struct GraphEntry {
        cudaGraphExec_t exec;
        int64_t launches;
    };
    std::map<std::vector<long long>, GraphEntry> gcache;
    // A captured graph holds the context buffers it copied to and from: when
    // one of them is reallocated (even at the same address) every graph is
    // dropped, since the CUDA driver may keep the old allocation's mapping in a
    // copy node.
    int64_t buf_gen = 0, graph_gen = 0;
    int64_t graphs_captured = 0, graph_replays = 0;
    // autotuner: engine, tile capacity and radix cap per batch shape
    struct Knobs {
        int fused, cap, maxr;
    };
    bool autotune = false;
    std::map<std::array<long long, 5>, Knobs> tuned;
    int64_t keys_tuned = 0;
    // caller's record of the device-resident searches' own evaluations
    double* rec = nullptr;
    int64_t rec_len = 0;
    int rec_cap = 0;
};

#include <chrono>
// wall time of a host phase, accumulated under "host:*" when profiling is on
struct HostTimer {
    kdefft_ctx c;
    const char* name;
    std::chrono::steady_clock::time_point t0;
    HostTimer(kdefft_ctx c_, const char* n) : c(c_), name(n), t0(std::chrono::steady_clock::now()) {}
    ~HostTimer() {
        if (!c->prof) return;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        auto& k = c->kstat[name];
        k.launches++;
        k.ms += ms;
    }
};

static cudaEvent_t ev_get(kdefft_ctx c) {
    if (!c->evpool.empty()) {
        cudaEvent_t e = c->evpool.back();
        c->evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket a launch: returns the start event (or null when profiling is off).
static cudaEvent_t prof_start(kdefft_ctx c) {
    c->launches++;
    if (!c->prof) return nullptr;
    cudaEvent_t a = ev_get(c);
    cudaEventRecord(a, c->stream);
    return a;
}

static void prof_stop(kdefft_ctx c, cudaEvent_t a, const char* name, double bytes, double flops) {
    if (!c->prof || !a) return;
    cudaEvent_t b = ev_get(c);
    cudaEventRecord(b, c->stream);
    c->pending.push_back({name, a, b, bytes, flops});
}

// after a stream synchronisation: fold the finished event pairs into the stats
static void prof_flush(kdefft_ctx c) {
    for (auto& p : c->pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);   // launches may still be in flight
        cudaEventElapsedTime(&ms, p.a, p.b);
        auto& k = c->kstat[p.name];
        k.launches++;
        k.ms += ms;
        k.bytes += p.bytes;
        k.flops += p.flops;
        c->evpool.push_back(p.a);
        c->evpool.push_back(p.b);
    }
    c->pending.clear();
}

// Destroy every cached graph once the work launched so far is done.
static int drop_graphs(kdefft_ctx c) {
    KCU(cudaStreamSynchronize(c->stream));
    for (auto& kv : c->gcache) cudaGraphExecDestroy(kv.second.exec);
    c->gcache.clear();
    return KDEFFT_OK;
}

// The pinned staging buffer h_items feeds one host-to-device copy per
// batch.  Before the host rewrites it, the previous copy out of it must be
// done: an event recorded right after that copy marks it (the kernels that
// follow may still run).
static int staging_wait(kdefft_ctx c) {
    if (!c->staging_free) {
        KCU(cudaEventSynchronize(c->staging_ev));
        c->staging_free = true;
    }
    return KDEFFT_OK;
}

static int staging_upload(kdefft_ctx c, void* dst, size_t bytes) {
    KCU(cudaMemcpyAsync(dst, c->h_items.p, bytes, cudaMemcpyHostToDevice, c->stream));
    KCU(cudaEventRecord(c->staging_ev, c->stream));
    c->staging_free = false;
    return KDEFFT_OK;
}

// Run the stream work of one batch (`issue`: the copies and launches it
// enqueues on c->stream) directly, or replay it from a CUDA graph cached
// under its launch signature `sig` (every pointer, size and launch shape the
// work depends on; the pinned staging buffers are read when the graph runs,
// so new contents need no new graph).  Direct while profiling, so that
// every kernel keeps its own CUDA events.
template <typename F>
static int run_graph(kdefft_ctx c, const std::vector<long long>& sig, F&& issue) {
    if (!c->graphs || c->prof) return issue();
    if (c->graph_gen != c->buf_gen) {   // a buffer some graph uses was reallocated
        if (!c->gcache.empty()) KCHK(drop_graphs(c));
        c->graph_gen = c->buf_gen;
    }
    auto it = c->gcache.find(sig);
    if (it == c->gcache.end()) {
        if (!c->cap_stream) KCU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        if (c->gcache.size() >= 64) KCHK(drop_graphs(c));
        // capture on the library's own stream (the caller's may be the legacy
        // default stream, which cannot be captured); replay on the caller's
        cudaStream_t user = c->stream;
        const int64_t l0 = c->launches;
        KCU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
        c->stream = c->cap_stream;
        const int r = issue();
        c->stream = user;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        if (r != KDEFFT_OK) {
            if (g) cudaGraphDestroy(g);
            c->launches = l0;
            return r;
        }
        KCU(e);
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        KCU(ei);
        if (c->graph_gen != c->buf_gen) {   // the capture itself reallocated a buffer: run it once, keep nothing
            const cudaError_t el = cudaGraphLaunch(ex, c->stream);
            const cudaError_t es = cudaStreamSynchronize(c->stream);
            cudaGraphExecDestroy(ex);
            KCU(el);
            KCU(es);
            return KDEFFT_OK;
        }
        it = c->gcache.emplace(sig, kdefft_ctx_s::GraphEntry{ex, c->launches - l0}).first;
        c->launches = l0;
        c->graphs_captured++;
    } else {
        c->graph_replays++;
    }
    c->launches += it->second.launches;
    KCU(cudaGraphLaunch(it->second.exec, c->stream));
    return KDEFFT_OK;
}

struct kdefft_ds_s {
    kdefft_ctx ctx = nullptr;
    int d = 0;
    int64_t n = 0;
    int64_t dropped = 0;
    double lo[4] = {0}, hi[4] = {0}, delta[4] = {0};
    int64_t M[4] = {1, 1, 1, 1};
    int64_t ncells = 0;
    kdefft_opts opts;
    DevBuf counts;        // float or double
    DevBuf counts_i;      // int32 (simple binning)
    DevBuf counts64;      // FP64 copy of FP32 counts, made on first FP64 use
    std::map<std::vector<int>, std::shared_ptr<DevBuf>> spectra;
    double cov[16] = {0}; // sample covariance (d x d, row-major)
    std::map<std::vector<double>, double> c2g;   // SCV phi_2G sums by (G, L, P)
    // count autocorrelation a_j on the half box A (lag-domain engine), FP64
    // and an FP32 copy
    int acA[4] = {-1, -1, -1, -1};
    DevBuf ac64, ac32;
    std::shared_ptr<DevBuf> pool;   // memory that `counts` views (datasets binned together share one)
};

// dataset buffers draw on the context's block cache
static void attach_cache(kdefft_ds_s& ds, kdefft_ctx c) {
    for (DevBuf* b : {&ds.counts, &ds.counts_i, &ds.counts64, &ds.ac64, &ds.ac32}) b->cache = &c->cache;
}

static int twiddle_offset(kdefft_ctx c, int P) {
    auto it = c->tw_off.find(P);
    if (it != c->tw_off.end()) return it->second;
    const int off = (int)(c->tw_host.size() / 2);
    for (int t = 0; t < P; ++t) {
        const long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)t / (long double)P;
        c->tw_host.push_back((double)cosl(ang));
        c->tw_host.push_back((double)sinl(ang));
    }
    c->tw_off[P] = off;
    return off;
}

// make every twiddle on the host resident on the device
static int sync_twiddles(kdefft_ctx c) {
    const size_t n = c->tw_host.size() / 2;
    if (n == c->tw_dev_n) return KDEFFT_OK;
    KCU(cudaStreamSynchronize(c->stream));
    KCHK(c->tw64.ensure(n * sizeof(double2)));
    KCHK(c->tw32.ensure(n * sizeof(float2)));
    KCHK(c->twdf.ensure(n * sizeof(double2)));
    std::vector<float> f(2 * n), fp(4 * n);
    for (size_t i = 0; i < 2 * n; ++i) {
        const double v = c->tw_host[i];
        f[i] = (float)v;
        fp[2 * i] = (float)v;                          // FP32 pair: leading part
        fp[2 * i + 1] = (float)(v - (double)(float)v);  // and its remainder
    }
    KCU(cudaMemcpy(c->tw64.p, c->tw_host.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
    KCU(cudaMemcpy(c->tw32.p, f.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
    KCU(cudaMemcpy(c->twdf.p, fp.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
    c->tw_dev_n = n;
    return KDEFFT_OK;
}

// ============================================================ kernel descriptions
struct Term {
    int sig;
    int alpha[MAXD];
    double w;   // weight of d^alpha phi_Sigma (the Hermite sign is applied later)
};

struct KSpec {
    int nsig = 0;
    Mat sig[MAXSIG];
};

// The terms of one grid: up to four held inline (no allocation per grid,
// which dominates building a request set of thousands of bandwidths), more
// in a vector.
class TermVec {
    static constexpr int kInline = 4;
    Term in_[kInline];
    int n_ = 0;
    std::vector<Term> ex_;   // all terms once there are more than kInline

public:
    TermVec() = default;
    TermVec(std::initializer_list<Term> l) { *this = l; }
    TermVec(const std::vector<Term>& v) { *this = v; }
    int size() const { return ex_.empty() ? n_ : (int)ex_.size(); }
    bool empty() const { return size() == 0; }
    const Term* begin() const { return ex_.empty() ? in_ : ex_.data(); }
    const Term* end() const { return begin() + size(); }
    const Term& operator[](int i) const { return begin()[i]; }
    void clear() {
        n_ = 0;
        ex_.clear();
    }
    void push_back(const Term& t) {
        if (ex_.empty() && n_ < kInline) {
            in_[n_++] = t;
            return;
        }
        if (ex_.empty()) ex_.assign(in_, in_ + n_);
        ex_.push_back(t);
    }
    void assign(int n, const Term& t) {
        clear();
        for (int i = 0; i < n; ++i) push_back(t);
    }
    TermVec& operator=(const std::vector<Term>& v) {
        clear();
        for (const Term& t : v) push_back(t);
        return *this;
    }
    TermVec& operator=(std::initializer_list<Term> l) {
        clear();
        for (const Term& t : l) push_back(t);
        return *this;
    }
};

// One real lag kernel to be reduced against a dataset's spectrum.
struct GridReq {
    kdefft_ds ds;
    int spec;              // index into the request set's KSpec list
    int L[4];
    int P[4];
    TermVec terms;
    bool fp64 = false;     // evaluate in FP64 even on an FP32 dataset
    double value = 0.0;    // result: n^-2 sum_w |C|^2 K / prod P  (= Eq. 25)
};

struct ReqSet {
    std::vector<KSpec> specs;
    std::vector<GridReq> grids;
};

static int support_L(const kdefft_ds ds, double lam, int* L) {
    for (int k = 0; k < ds->d; ++k) {
        const double v = ds->opts.tau * std::sqrt(std::fabs(lam)) / ds->delta[k];
        double c = std::ceil(v);
        const double cap = (double)(ds->M[k] - 1);
        if (!(c <= cap)) c = cap;   // also catches NaN/inf
        if (c < 1.0) c = 1.0;
        L[k] = (int)c;
    }
    return KDEFFT_OK;
}

static int choose_P(const kdefft_ds ds, const int* L, int* P) {
    for (int k = 0; k < ds->d; ++k) {
        const long long M = ds->M[k];
        long long p = 0;
        switch (ds->opts.P_rule) {
            case KDEFFT_P_PAPER: {
                p = 1;
                while (p < M + 2 * L[k] - 1) p *= 2;
                break;
            }
            case KDEFFT_P_PAPER_FULL: {
                p = 1;
                while (p < 3 * M - 1) p *= 2;
                break;
            }
            case KDEFFT_P_FIXED:
                p = ds->opts.P_fixed[k];
                break;
            default: {
                p = next_smooth(M + L[k]);
            }
        }
        if (p < M + L[k]) return fail(KDEFFT_ERR_ARG, "padded size P_k below M_k + L_k would alias");
        if (p > MAXP || !is_smooth(p))
            return fail(KDEFFT_ERR_UNSUPPORTED, "padded size " + std::to_string(p) + " not 2^a3^b5^c <= 4096");
        P[k] = (int)p;
    }
    return KDEFFT_OK;
}

// support and padding for a kernel whose basis matrix is B
// lambda_max in closed form for d <= 3 (d = 2: the larger root of the
// characteristic quadratic; d = 3: the trigonometric solution of the
// characteristic cubic of a symmetric matrix), Jacobi otherwise
static double lambda_max_closed(const Mat& S) {
    const int d = S.d;
    if (d == 1) return S(0, 0);
    if (d == 2) {
        const double h = 0.5 * (S(0, 0) - S(1, 1));
        return 0.5 * (S(0, 0) + S(1, 1)) + std::sqrt(h * h + S(0, 1) * S(0, 1));
    }
    if (d == 3) {
        const double p1 = S(0, 1) * S(0, 1) + S(0, 2) * S(0, 2) + S(1, 2) * S(1, 2);
        if (p1 == 0.0) return std::max(S(0, 0), std::max(S(1, 1), S(2, 2)));
        const double q = (S(0, 0) + S(1, 1) + S(2, 2)) / 3.0;
        const double a = S(0, 0) - q, b = S(1, 1) - q, c = S(2, 2) - q;
        const double p = std::sqrt((a * a + b * b + c * c + 2.0 * p1) / 6.0);
        // det((S - q I) / p) / 2, clamped to the cosine's range
        const double B01 = S(0, 1) / p, B02 = S(0, 2) / p, B12 = S(1, 2) / p, Ba = a / p, Bb = b / p, Bc = c / p;
        double r = 0.5 * (Ba * (Bb * Bc - B12 * B12) - B01 * (B01 * Bc - B12 * B02) + B02 * (B01 * B12 - Bb * B02));
        r = std::min(1.0, std::max(-1.0, r));
        return q + 2.0 * p * std::cos(std::acos(r) / 3.0);
    }
    return lambda_max(S);
}

// The support of Eq. 26 from lambda_max of B: the closed form first; where
// tau sqrt(lambda) / delta_k falls within 1e-7 (relative) of an integer, the
// support could round the other way, so lambda comes from the Jacobi
// rotations instead (machine precision).  The closed form costs a tenth of
// the rotations: the supports of a batch of many bandwidths.
static int plan_for(const kdefft_ds ds, const Mat& B, int* L, int* P) {
    if (ds->opts.L_basis == KDEFFT_L_FULL) {
        for (int k = 0; k < ds->d; ++k) L[k] = (int)(ds->M[k] - 1);
    } else {
        double lam = lambda_max_closed(B);
        bool near = !std::isfinite(lam);
        for (int k = 0; k < ds->d && !near; ++k) {
            const double v = ds->opts.tau * std::sqrt(std::fabs(lam)) / ds->delta[k];
            near = std::fabs(v - std::nearbyint(v)) <= 1e-7 * std::max(1.0, std::fabs(v));
        }
        if (near) lam = lambda_max(B);
        KCHK(support_L(ds, lam, L));
    }
    return choose_P(ds, L, P);
}

static int spd_or_fail(const Mat& S, const char* what) {
    Mat L;
    if (!cholesky(S, L)) return fail(KDEFFT_ERR_NOT_SPD, std::string(what) + " is not positive definite");
    return KDEFFT_OK;
}

static void alpha2(int d, int a, int b, int* out) {
    for (int k = 0; k < MAXD; ++k) out[k] = 0;
    out[a] += 1;
    out[b] += 1;
    (void)d;
}

// ---- LSCV (Eqs. 8, 10-11) ------------------------------------------------
// grids: [value grids..., gradient grids (a <= b)...]
// grids of one LSCV bandwidth: the value grid(s), then the gradient grids
static int lscv_grid_count(kdefft_ds ds, bool grad) {
    const int d = ds->d;
    return (ds->opts.exact_loo ? 2 : 1) + (grad ? d * (d + 1) / 2 : 0);
}

// The LSCV requests of one bandwidth written in place: its kernel spec at
// rs.specs[si], its grids at rs.grids[g0 ..] (lscv_grid_count of them).
static int add_lscv_at(ReqSet& rs, kdefft_ds ds, const Mat& H, bool grad, int si, int g0) {
    const int d = ds->d;
    KCHK(spd_or_fail(H, "H"));
    KSpec& sp = rs.specs[si];
    sp.nsig = 2;
    sp.sig[0] = scaled(2.0, H);
    sp.sig[1] = H;
    int L[4], P[4];
    const Mat& basis = (ds->opts.L_basis == KDEFFT_L_WIDEST) ? sp.sig[0] : H;
    KCHK(plan_for(ds, basis, L, P));
    int gi = g0;
    auto put = [&](TermVec t) {
        GridReq& g = rs.grids[gi++];
        g.ds = ds;
        g.spec = si;
        std::memcpy(g.L, L, sizeof(L));
        std::memcpy(g.P, P, sizeof(P));
        g.terms = std::move(t);
    };
    const double n = (double)ds->n;
    if (!ds->opts.exact_loo) {
        put({Term{0, {0, 0, 0, 0}, 1.0}, Term{1, {0, 0, 0, 0}, -2.0}});
    } else {
        put({Term{0, {0, 0, 0, 0}, 1.0}});
        put({Term{1, {0, 0, 0, 0}, 1.0}});
    }
    if (grad) {
        const double f = ds->opts.exact_loo ? n / (n - 1.0) : 1.0;
        for (int a = 0; a < d; ++a)
            for (int b = a; b < d; ++b) {
                const double s = (a == b) ? 1.0 : 2.0;
                Term t0{0, {0}, s}, t1{1, {0}, -s * f};
                alpha2(d, a, b, t0.alpha);
                alpha2(d, a, b, t1.alpha);
                put({t0, t1});
            }
    }
    return KDEFFT_OK;
}

// grids: [value grids..., gradient grids (a <= b)...]
static int add_lscv(ReqSet& rs, kdefft_ds ds, const Mat& H, bool grad, int& first) {
    const int si = (int)rs.specs.size();
    first = (int)rs.grids.size();
    rs.specs.emplace_back();
    rs.grids.resize(rs.grids.size() + lscv_grid_count(ds, grad));
    return add_lscv_at(rs, ds, H, grad, si, first);
}

// The LSCV requests of many bandwidths (owner[h]: the dataset of H_h): the
// layout first, then the bandwidths over index ranges that may run on
// several host threads.  On a failure the set is rebuilt serially, which
// reports it exactly.
static int add_lscv_many(ReqSet& rs, const std::vector<kdefft_ds>& owner, const std::vector<Mat>& Hs, bool grad,
                         std::vector<int>& first) {
    const size_t nt = Hs.size();
    const size_t s0 = rs.specs.size(), g00 = rs.grids.size();
    first.assign(nt, 0);
    size_t ng = g00;
    for (size_t h = 0; h < nt; ++h) {
        first[h] = (int)ng;
        ng += lscv_grid_count(owner[h], grad);
    }
    rs.specs.resize(s0 + nt);
    rs.grids.resize(ng);
    std::atomic<int> err{KDEFFT_OK};
    host_parallel_for(nt, 2048, [&](size_t h0, size_t h1) {
        for (size_t h = h0; h < h1 && err == KDEFFT_OK; ++h)
            if (add_lscv_at(rs, owner[h], Hs[h], grad, (int)(s0 + h), first[h]) != KDEFFT_OK) err = KDEFFT_ERR_ARG;
    });
    if (err == KDEFFT_OK) return KDEFFT_OK;
    rs.specs.resize(s0);
    rs.grids.resize(g00);
    for (size_t h = 0; h < nt; ++h) KCHK(add_lscv(rs, owner[h], Hs[h], grad, first[h]));
    return KDEFFT_OK;
}

// ---- SCV (reading; Gaussian pilot G) --------------------------------------
// split64: the value as two FP64 Gaussian sums (plus the cached phi_2G sum)
// combined in FP64; otherwise one FP32 grid of the whole SCV kernel.
static int add_scv(ReqSet& rs, kdefft_ds ds, const Mat& H, const Mat& G, bool grad, bool split64, int& first) {
    const int d = ds->d;
    KCHK(spd_or_fail(H, "H"));
    KSpec sp;
    sp.nsig = 3;
    sp.sig[0] = lin(2.0, H, 2.0, G);
    sp.sig[1] = lin(1.0, H, 2.0, G);
    sp.sig[2] = scaled(2.0, G);
    const int si = (int)rs.specs.size();
    rs.specs.push_back(sp);
    int L[4], P[4];
    const Mat& basis = (ds->opts.L_basis == KDEFFT_L_PAPER) ? H : sp.sig[0];
    KCHK(plan_for(ds, basis, L, P));
    first = (int)rs.grids.size();
    auto push = [&](TermVec t) {
        GridReq g;
        g.ds = ds;
        g.spec = si;
        std::memcpy(g.L, L, sizeof(L));
        std::memcpy(g.P, P, sizeof(P));
        g.terms = std::move(t);
        rs.grids.push_back(std::move(g));
    };
    // value: the two H-dependent Gaussians as separate grids (one packed pair);
    // their difference and the H-independent phi_2G sum are combined in FP64,
    // because the full SCV kernel integrates to zero and its transform near
    // w = 0 would cancel in FP32
    if (split64) {
        push({Term{0, {0}, 1.0}});
        push({Term{1, {0}, 1.0}});
        rs.grids[first].fp64 = rs.grids[first + 1].fp64 = true;
    } else {
        push({Term{0, {0}, 1.0}, Term{1, {0}, -2.0}, Term{2, {0}, 1.0}});
    }
    if (grad) {
        for (int a = 0; a < d; ++a)
            for (int b = a; b < d; ++b) {
                const double s = (a == b) ? 1.0 : 2.0;
                Term t0{0, {0}, s}, t1{1, {0}, -s};
                alpha2(d, a, b, t0.alpha);
                alpha2(d, a, b, t1.alpha);
                push({t0, t1});
            }
    }
    return KDEFFT_OK;
}

// ---- psi_r (Eq. 13): one grid per unique multi-index |alpha| = r ----------
// the multi-indices alpha with |alpha| = r in graded order (the unique
// partials of psi_r)
static std::vector<MultiIndex> order_alphas(int d, int r) {
    std::vector<MultiIndex> alphas;
    for (const MultiIndex& m : hindex().list[d]) {
        int o = 0;
        for (int k = 0; k < d; ++k) o += m.a[k];
        if (o == r) alphas.push_back(m);
    }
    return alphas;
}

// The psi_r requests of one bandwidth written in place: its spec at
// rs.specs[si], one grid per partial at rs.grids[g0 ..].
static int add_psi_at(ReqSet& rs, kdefft_ds ds, const Mat& H, const std::vector<MultiIndex>& alphas, int si,
                      int g0) {
    const int d = ds->d;
    KSpec& sp = rs.specs[si];
    sp.nsig = 1;
    sp.sig[0] = H;
    int L[4], P[4];
    KCHK(plan_for(ds, H, L, P));
    int gi = g0;
    for (const MultiIndex& m : alphas) {
        GridReq& g = rs.grids[gi++];
        g.ds = ds;
        g.spec = si;
        std::memcpy(g.L, L, sizeof(L));
        std::memcpy(g.P, P, sizeof(P));
        Term t{0, {0}, 1.0};
        for (int k = 0; k < MAXD; ++k) t.alpha[k] = (k < d) ? m.a[k] : 0;
        g.terms.assign(1, t);
    }
    return KDEFFT_OK;
}

static int add_psi(ReqSet& rs, kdefft_ds ds, const Mat& H, const std::vector<MultiIndex>& alphas, int& first) {
    const int si = (int)rs.specs.size();
    first = (int)rs.grids.size();
    rs.specs.emplace_back();
    rs.grids.resize(rs.grids.size() + alphas.size());
    return add_psi_at(rs, ds, H, alphas, si, first);
}

// psi_r requests of many bandwidths of one dataset: checks and layout
// first, then the bandwidths over index ranges that may run on several host
// threads; on a failure the set is rebuilt serially (exact report).
static int add_psi_many(ReqSet& rs, kdefft_ds ds, const std::vector<Mat>& Hs, const std::vector<MultiIndex>& alphas,
                        std::vector<int>& first) {
    const size_t nH = Hs.size(), na = alphas.size();
    const size_t s0 = rs.specs.size(), g00 = rs.grids.size();
    first.assign(nH, 0);
    for (size_t h = 0; h < nH; ++h) first[h] = (int)(g00 + h * na);
    rs.specs.resize(s0 + nH);
    rs.grids.resize(g00 + nH * na);
    std::atomic<int> err{KDEFFT_OK};
    host_parallel_for(nH, 1024, [&](size_t h0, size_t h1) {
        for (size_t h = h0; h < h1 && err == KDEFFT_OK; ++h)
            if (add_psi_at(rs, ds, Hs[h], alphas, (int)(s0 + h), first[h]) != KDEFFT_OK) err = KDEFFT_ERR_ARG;
    });
    if (err == KDEFFT_OK) return KDEFFT_OK;
    rs.specs.resize(s0);
    rs.grids.resize(g00);
    for (size_t h = 0; h < nH; ++h) KCHK(add_psi(rs, ds, Hs[h], alphas, first[h]));
    return KDEFFT_OK;
}

// ---- eta_{0,2}(x; B, Sigma) = (vec^T B)^{(x)2} D^{(x)4} phi_Sigma (Eq. 30) ----
// ---- eta_m (Eq. 31), Q_r (Eq. 32), LSCV_r (Eqs. 35-36) --------------------
// eta_m(x; Sigma) = (vec^T I)^{(x)m} D^{(x)2m} phi_Sigma = Laplacian^m phi_Sigma
//                 = sum_{|beta| = m} m! / beta! d^{2 beta} phi_Sigma,
// appended as terms of covariance `sig` scaled by `scale`.
template <typename V>
static void laplacian_power_terms(int d, int m, int sig, double scale, V& out) {
    std::vector<MultiIndex> all;
    enumerate(d, m, all);
    double mf = 1.0;
    for (int i = 2; i <= m; ++i) mf *= i;
    for (const MultiIndex& b : all) {
        int o = 0;
        double den = 1.0;
        for (int k = 0; k < d; ++k) {
            o += b.a[k];
            for (int i = 2; i <= b.a[k]; ++i) den *= i;
        }
        if (o != m) continue;
        Term t{sig, {0, 0, 0, 0}, scale * mf / den};
        for (int k = 0; k < d; ++k) t.alpha[k] = 2 * b.a[k];
        out.push_back(t);
    }
}

// d^alpha phi_Sigma at x = 0: (-1)^{|alpha|} He_alpha(0; Lambda) phi_Sigma(0),
// He_0 = 1, He_{beta + e_i}(0) = -sum_j beta_j Lambda_ij He_{beta - e_j}(0)
// (the Hermite recurrence of the kernels at z = 0), FP64.
static double dphi_at0(const Mat& Sigma, const int* alpha) {
    const int d = Sigma.d;
    Mat inv;
    double det;
    spd_inv_det(Sigma, inv, det);
    std::map<std::vector<int>, double> memo;
    std::function<double(const std::vector<int>&)> he = [&](const std::vector<int>& a) -> double {
        int tot = 0;
        for (int v : a) tot += v;
        if (tot == 0) return 1.0;
        auto it = memo.find(a);
        if (it != memo.end()) return it->second;
        int i = 0;
        while (a[i] == 0) ++i;
        std::vector<int> b = a;
        b[i]--;
        double v = 0.0;
        for (int j = 0; j < d; ++j)
            if (b[j] > 0) {
                std::vector<int> c = b;
                c[j]--;
                v -= b[j] * inv(i, j) * he(c);
            }
        memo[a] = v;
        return v;
    };
    std::vector<int> a(alpha, alpha + d);
    int tot = 0;
    for (int v : a) tot += v;
    const double phi0 = std::pow(2.0 * M_PI, -0.5 * d) / std::sqrt(det);
    return ((tot & 1) ? -1.0 : 1.0) * he(a) * phi0;
}

// one grid: eta_m(.; Sigma) with support from lambda_max(Sigma)
static int add_eta_m(ReqSet& rs, kdefft_ds ds, const Mat& Sg, int m, int& first) {
    KCHK(spd_or_fail(Sg, "Sigma"));
    KSpec sp;
    sp.nsig = 1;
    sp.sig[0] = Sg;
    const int si = (int)rs.specs.size();
    rs.specs.push_back(sp);
    int L[4], P[4];
    KCHK(plan_for(ds, Sg, L, P));
    first = (int)rs.grids.size();
    GridReq g;
    g.ds = ds;
    g.spec = si;
    std::memcpy(g.L, L, sizeof(L));
    std::memcpy(g.P, P, sizeof(P));
    laplacian_power_terms(ds->d, m, 0, 1.0, g.terms);
    rs.grids.push_back(std::move(g));
    return KDEFFT_OK;
}

// LSCV_r grids: Eq. 36 one grid eta_r(.; 2H) - 2 eta_r(.; H); Eq. 35 (exact
// leave-one-out) the two sums separately
static int add_lscv_r(ReqSet& rs, kdefft_ds ds, const Mat& H, int r, int& first) {
    KCHK(spd_or_fail(H, "H"));
    KSpec sp;
    sp.nsig = 2;
    sp.sig[0] = scaled(2.0, H);
    sp.sig[1] = H;
    const int si = (int)rs.specs.size();
    rs.specs.push_back(sp);
    int L[4], P[4];
    const Mat& basis = (ds->opts.L_basis == KDEFFT_L_WIDEST) ? sp.sig[0] : H;
    KCHK(plan_for(ds, basis, L, P));
    first = (int)rs.grids.size();
    auto push = [&](TermVec t) {
        GridReq g;
        g.ds = ds;
        g.spec = si;
        std::memcpy(g.L, L, sizeof(L));
        std::memcpy(g.P, P, sizeof(P));
        g.terms = std::move(t);
        rs.grids.push_back(std::move(g));
    };
    std::vector<Term> a, b;
    if (!ds->opts.exact_loo) {
        laplacian_power_terms(ds->d, r, 0, 1.0, a);
        laplacian_power_terms(ds->d, r, 1, -2.0, a);
        push(a);
    } else {
        laplacian_power_terms(ds->d, r, 0, 1.0, a);
        laplacian_power_terms(ds->d, r, 1, 1.0, b);
        push(a);
        push(b);
    }
    return KDEFFT_OK;
}

// eta_{r,s}(x; A, B, Sigma) = {(vec^T A)^{(x)r} (x) (vec^T B)^{(x)s}} D^{(x)2r+2s} phi_Sigma
// (Eq. 30): the sum over index tuples of prod A_{pair} prod B_{pair} times the
// derivative along the tuple, collected by multi-index; support from
// lambda_max(Sigma)
static int add_eta_rs(ReqSet& rs, kdefft_ds ds, const Mat& A, const Mat& B, const Mat& Sg, int r, int s, int& first) {
    const int d = ds->d;
    KCHK(spd_or_fail(Sg, "Sigma"));
    KSpec sp;
    sp.nsig = 1;
    sp.sig[0] = Sg;
    const int si = (int)rs.specs.size();
    rs.specs.push_back(sp);
    int L[4], P[4];
    KCHK(plan_for(ds, Sg, L, P));
    first = (int)rs.grids.size();
    std::map<std::vector<int>, double> w;
    std::vector<int> al(MAXD, 0);
    std::function<void(int, double)> pairs = [&](int k, double c) {
        if (c == 0.0) return;
        if (k == r + s) {
            w[al] += c;
            return;
        }
        const Mat& M = (k < r) ? A : B;
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                al[a]++;
                al[b]++;
                pairs(k + 1, c * M(a, b));
                al[a]--;
                al[b]--;
            }
    };
    pairs(0, 1.0);
    GridReq g;
    g.ds = ds;
    g.spec = si;
    std::memcpy(g.L, L, sizeof(L));
    std::memcpy(g.P, P, sizeof(P));
    for (auto& kv : w) {
        if (kv.second == 0.0) continue;
        Term t{0, {0, 0, 0, 0}, kv.second};
        for (int k = 0; k < MAXD; ++k) t.alpha[k] = kv.first[k];
        g.terms.push_back(t);
    }
    if ((int)g.terms.size() > MAXTERM) return fail(KDEFFT_ERR_UNSUPPORTED, "too many kernel terms");
    rs.grids.push_back(std::move(g));
    return KDEFFT_OK;
}

static int add_eta02(ReqSet& rs, kdefft_ds ds, const Mat& B, const Mat& Sg, int& first) {
    const int d = ds->d;
    KSpec sp;
    sp.nsig = 1;
    sp.sig[0] = Sg;
    const int si = (int)rs.specs.size();
    rs.specs.push_back(sp);
    int L[4], P[4];
    KCHK(plan_for(ds, Sg, L, P));
    first = (int)rs.grids.size();
    std::map<std::vector<int>, double> w;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b)
            for (int c = 0; c < d; ++c)
                for (int e = 0; e < d; ++e) {
                    std::vector<int> al(MAXD, 0);
                    al[a]++;
                    al[b]++;
                    al[c]++;
                    al[e]++;
                    w[al] += B(a, b) * B(c, e);
                }
    GridReq g;
    g.ds = ds;
    g.spec = si;
    std::memcpy(g.L, L, sizeof(L));
    std::memcpy(g.P, P, sizeof(P));
    for (auto& kv : w) {
        if (kv.second == 0.0) continue;
        Term t{0, {0}, kv.second};
        for (int k = 0; k < MAXD; ++k) t.alpha[k] = kv.first[k];
        g.terms.push_back(t);
    }
    rs.grids.push_back(std::move(g));
    return KDEFFT_OK;
}

// ============================================================ execution
static size_t spec_elems(int d, const int* P) {
    size_t q = (size_t)(P[d - 1] / 2 + 1);
    for (int k = 0; k < d - 1; ++k) q *= (size_t)P[k];
    return q;
}

template <typename real>
static int fill_axes(kdefft_ctx c, int d, const int* P, Item<real>& it, int maxr = 0) {
    if (maxr <= 0) maxr = sizeof(real) == 8 ? 16 : 32;
    for (int k = 0; k < d; ++k) {
        if (!radix_plan(P[k], it.ax[k], maxr))
            return fail(KDEFFT_ERR_UNSUPPORTED, "no radix plan for P");
        it.ax[k].tw_off = twiddle_offset(c, P[k]);
    }
    return KDEFFT_OK;
}

// Tiles and scratch of one item; appends to the per-pass tile lists.
struct PassLists {
    std::vector<Tile> A, mid[MAXD], F;
    int capA = 0, capM[MAXD] = {0}, capF = 0;
    int pA = 0, pM[MAXD] = {0}, pF = 0;
    long long scratch = 0;
};

// complex scratch elements an item needs (both ping-pong regions)
template <typename real>
static long long scratch_need(const Item<real>& it) {
    const int d = it.d;
    long long linesA = 1;
    for (int k = 0; k < d - 1; ++k) linesA *= it.S[k];
    long long sz[2] = {(d >= 2) ? (long long)(it.ax[d - 1].P / 2 + 1) * linesA : 0, 0};
    long long Wo = it.ax[d - 1].P / 2 + 1;
    int wsel = 0;
    for (int k = d - 2; k >= 1; --k) {
        long long O = 1;
        for (int m = 0; m < k; ++m) O *= it.S[m];
        Wo *= it.ax[k].P;
        wsel ^= 1;
        sz[wsel] = std::max(sz[wsel], Wo * O);
    }
    return sz[0] + sz[1];
}

template <typename real>
static void tile_item(Item<real>& it, int idx, int cap, PassLists& pl) {
    const int d = it.d;
    const int Pl = it.ax[d - 1].P;
    const int Ql = Pl / 2 + 1;
    long long linesA = 1;
    for (int k = 0; k < d - 1; ++k) linesA *= it.S[k];
    // stage A
    {
        const int nl = std::max(1, std::min<int>(cap / Pl, (int)linesA));
        for (long long l0 = 0; l0 < linesA; l0 += nl) {
            const int n = (int)std::min<long long>(nl, linesA - l0);
            pl.A.push_back(Tile{idx, (int)l0, 0, n});
            pl.capA = std::max(pl.capA, n * Pl);
        }
        pl.pA = std::max(pl.pA, Pl);
    }
    // scratch sizes (two ping-pong regions)
    long long sz[2] = {0, 0};
    long long cur = (d >= 2) ? (long long)Ql * linesA : 0;
    sz[0] = cur;
    int wsel = 0;
    long long Wo = Ql;   // transformed outer extent
    for (int k = d - 2; k >= 1; --k) {
        long long O = 1;
        for (int m = 0; m < k; ++m) O *= it.S[m];
        const int Pk = it.ax[k].P;
        const int nl = std::max(1, std::min<int>(cap / Pk, (int)O));
        for (long long wo = 0; wo < Wo; ++wo)
            for (long long o0 = 0; o0 < O; o0 += nl) {
                const int n = (int)std::min<long long>(nl, O - o0);
                pl.mid[k].push_back(Tile{idx, (int)wo, (int)o0, n});
                pl.capM[k] = std::max(pl.capM[k], n * Pk);
            }
        pl.pM[k] = std::max(pl.pM[k], Pk);
        Wo *= Pk;
        wsel ^= 1;
        sz[wsel] = std::max(sz[wsel], Wo * O);
    }
    it.scr[0] = pl.scratch;
    it.scr[1] = pl.scratch + sz[0];
    pl.scratch += sz[0] + sz[1];
    // final pass over q in [0, Wo)
    if (d >= 2) {
        const int P0 = it.ax[0].P;
        const int nl = std::max(1, std::min<int>(cap / P0, (int)Wo));
        it.tileF0 = (int)pl.F.size();
        int cnt = 0;
        for (long long q0 = 0; q0 < Wo; q0 += nl) {
            const int n = (int)std::min<long long>(nl, Wo - q0);
            pl.F.push_back(Tile{idx, (int)q0, 0, n});
            pl.capF = std::max(pl.capF, n * P0);
            ++cnt;
        }
        it.ntileF = cnt;
        pl.pF = std::max(pl.pF, P0);
    }
}

// Wait for the pending lag-domain results and store them in their requests.
static int flush_reads(kdefft_ctx c) {
    if (c->pend_reads.empty()) return KDEFFT_OK;
    {
        HostTimer w(c, "host:wait");
        KCU(cudaStreamSynchronize(c->stream));
    }
    const double* o = (const double*)c->h_out.p;
    for (const auto& pr : c->pend_reads)
        for (size_t i = 0; i < pr.pairs.size(); ++i) {
            pr.rs->grids[pr.pairs[i].first].value = o[pr.off + 2 * i];
            if (pr.pairs[i].second >= 0) pr.rs->grids[pr.pairs[i].second].value = o[pr.off + 2 * i + 1];
        }
    c->pend_reads.clear();
    c->hout_used = 0;
    return KDEFFT_OK;
}

template <typename real>
static int launch_items(kdefft_ctx c, std::vector<Item<real>>& items, PassLists& pl, int d, double* out_host) {
    using C = typename Cpx<real>::T;
    const int nitems = (int)items.size();
    if (nitems == 0) return KDEFFT_OK;
    if (out_host) KCHK(flush_reads(c));   // h_out is about to be rewritten
    KCHK(sync_twiddles(c));
    // d = 1: the single stage-A tile of each item owns partial slot tileF0
    if (d == 1) {
        for (int i = 0; i < nitems; ++i) {
            items[i].tileF0 = i;
            items[i].ntileF = 1;
        }
    }
    const size_t nF = (d == 1) ? (size_t)nitems : pl.F.size();
    // upload items + tiles in one copy
    const size_t bItems = sizeof(Item<real>) * nitems;
    const size_t nt = pl.A.size() + pl.F.size() + [&] {
        size_t s = 0;
        for (int k = 0; k < MAXD; ++k) s += pl.mid[k].size();
        return s;
    }();
    const size_t bTiles = sizeof(Tile) * nt;
    const size_t bytes = bItems + bTiles;
    // the pinned staging buffer may still be read by a previous copy (also
    // before it is reallocated)
    KCHK(staging_wait(c));
    KCHK(c->h_items.ensure(bytes));
    KCHK(c->items.ensure(bytes));
    unsigned char* h = (unsigned char*)c->h_items.p;
    std::memcpy(h, items.data(), bItems);
    size_t o = bItems;
    auto put = [&](const std::vector<Tile>& v) {
        const size_t first = (o - bItems) / sizeof(Tile);
        if (!v.empty()) std::memcpy(h + o, v.data(), sizeof(Tile) * v.size());
        o += sizeof(Tile) * v.size();
        return first;
    };
    const size_t offA = put(pl.A);
    size_t offM[MAXD];
    for (int k = 0; k < MAXD; ++k) offM[k] = put(pl.mid[k]);
    const size_t offF = put(pl.F);
    const Item<real>* dItems = (const Item<real>*)c->items.p;
    const Tile* dTiles = (const Tile*)((unsigned char*)c->items.p + bItems);
    KCHK(c->scratch.ensure(sizeof(C) * (size_t)std::max<long long>(pl.scratch, 1)));
    KCHK(c->partial.ensure(sizeof(double) * 2 * std::max<size_t>(nF, 1)));
    KCHK(c->out.ensure(sizeof(double) * 2 * nitems));
    C* scr = (C*)c->scratch.p;
    const C* tw = (const C*)(sizeof(real) == 4 ? c->tw32.p : c->tw64.p);
    double* part = (double*)c->partial.p;
    auto grid_of = [&](size_t ntiles) { return (int)std::min<size_t>(ntiles, (size_t)c->nsm * 4); };
    // algorithmic bytes and FFT flops (5 P log2 P per line) of each pass
    const double cs = (double)sizeof(C), rsz = (double)sizeof(real);
    auto fft_flops = [](double P) { return 5.0 * P * std::log2(P); };
    double bA = 0, fA = 0, bF = 0, fF = 0, bM[MAXD] = {0}, fM[MAXD] = {0};
    for (const Tile& t : pl.A) {
        const Item<real>& it = items[t.item];
        const double P = it.ax[d - 1].P, Q = std::floor(P / 2) + 1;
        fA += t.n * fft_flops(P);
        if (it.kind == 1) bA += t.n * it.S[d - 1] * rsz;            // counts read
        bA += (d == 1) ? Q * rsz : t.n * Q * cs;                      // spectrum read / half lines written
    }
    for (int k = 1; k <= d - 2; ++k)
        for (const Tile& t : pl.mid[k]) {
            const Item<real>& it = items[t.item];
            const double P = it.ax[k].P;
            fM[k] += t.n * fft_flops(P);
            bM[k] += t.n * (it.S[k] + P) * cs;
        }
    for (const Tile& t : pl.F) {
        const Item<real>& it = items[t.item];
        const double P = it.ax[0].P;
        fF += t.n * (fft_flops(P) + 4.0 * P);
        bF += t.n * (it.S[0] * cs + P * rsz);
    }
    std::vector<long long> sig = {1,
                                  (long long)sizeof(real),
                                  d,
                                  nitems,
                                  out_host ? 1 : 0,
                                  (long long)(uintptr_t)c->items.p,
                                  (long long)(uintptr_t)h,
                                  (long long)bytes,
                                  (long long)(uintptr_t)scr,
                                  (long long)(uintptr_t)tw,
                                  (long long)(uintptr_t)part,
                                  (long long)(uintptr_t)c->out.p,
                                  (long long)(uintptr_t)c->h_out.p,
                                  (long long)pl.A.size(),
                                  pl.pA,
                                  pl.capA,
                                  (long long)offA,
                                  (long long)pl.F.size(),
                                  pl.pF,
                                  pl.capF,
                                  (long long)offF};
    for (int k = 0; k < MAXD; ++k) {
        sig.push_back((long long)pl.mid[k].size());
        sig.push_back(pl.pM[k]);
        sig.push_back(pl.capM[k]);
        sig.push_back((long long)offM[k]);
    }
    if (out_host) KCHK(c->h_out.ensure(sizeof(double) * 2 * nitems));
    sig[12] = (long long)(uintptr_t)c->h_out.p;
    auto issue = [&]() -> int {
        cudaEvent_t ev;
        if (!pl.A.empty()) {
            ev = prof_start(c);
            KCU(launch_stage_a<real>(dItems, dTiles + offA, (int)pl.A.size(), pl.pA, pl.capA, scr, tw, part,
                                     grid_of(pl.A.size()), c->stream));
            prof_stop(c, ev, sizeof(real) == 4 ? "stage_a_f32" : "stage_a_f64", bA, fA);
        }
        for (int k = d - 2; k >= 1; --k)
            if (!pl.mid[k].empty()) {
                ev = prof_start(c);
                KCU(launch_mid<real>(dItems, dTiles + offM[k], (int)pl.mid[k].size(), k, pl.pM[k], pl.capM[k], scr,
                                     tw, grid_of(pl.mid[k].size()), c->stream));
                prof_stop(c, ev, sizeof(real) == 4 ? "mid_f32" : "mid_f64", bM[k], fM[k]);
            }
        if (d >= 2 && !pl.F.empty()) {
            ev = prof_start(c);
            KCU(launch_final<real>(dItems, dTiles + offF, (int)pl.F.size(), pl.pF, pl.capF, scr, tw, part,
                                   grid_of(pl.F.size()), c->stream));
            prof_stop(c, ev, sizeof(real) == 4 ? "final_f32" : "final_f64", bF, fF);
        }
        if (out_host) {
            ev = prof_start(c);
            KCU(launch_reduce<real>(dItems, nitems, part, (double*)c->out.p, c->stream));
            prof_stop(c, ev, "reduce", 16.0 * nF, 2.0 * nF);
            KCU(cudaMemcpyAsync(c->h_out.p, c->out.p, sizeof(double) * 2 * nitems, cudaMemcpyDeviceToHost, c->stream));
        }
        return KDEFFT_OK;
    };
    KCHK(staging_upload(c, c->items.p, bytes));
    KCHK(run_graph(c, sig, issue));
    c->h2d += (int64_t)bytes;
    if (out_host) {
        {
            HostTimer w(c, "host:wait");
            KCU(cudaStreamSynchronize(c->stream));
        }
        c->d2h += (int64_t)(sizeof(double) * 2 * nitems);
        std::memcpy(out_host, c->h_out.p, sizeof(double) * 2 * nitems);
        c->staging_free = true;
    }
    // without host results (count spectra) the launches stay in flight; the
    // next user of the staging buffer waits for the copy out of it
    prof_flush(c);
    return KDEFFT_OK;
}

static int cap_elems(bool dbl) { return dbl ? 3072 : 6144; }

// read and clear the device error flag (after a stream synchronisation)
static int check_errflag(kdefft_ctx c) {
    int h = 0;
    KCU(cudaMemcpy(&h, c->errflag, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        KCU(cudaMemset(c->errflag, 0, sizeof(int)));
        return fail(KDEFFT_ERR_TIMEOUT, "a device-side wait for a bulk copy timed out");
    }
    return KDEFFT_OK;
}

// d = 2, kernel items only: one cluster launch does every pass and the
// reduction.  Returns KDEFFT_ERR_UNSUPPORTED (without launching) when the
// items do not fit in shared memory for any cluster size; the caller then
// takes the multi-pass path.
template <typename real>
static int launch_fused(kdefft_ctx c, std::vector<Item<real>>& items, double* out_host) {
    using C = typename Cpx<real>::T;
    const int nitems = (int)items.size();
    KCHK(flush_reads(c));   // h_out is about to be rewritten
    const size_t budget = 200 * 1024;
    int rmax = 0;
    for (const Item<real>& it : items) rmax = std::max(rmax, it.R);
    if (rmax > 4 || (sizeof(real) == 8 && rmax > 2)) return KDEFFT_ERR_UNSUPPORTED;
    int cs = 2;
    while (cs < c->max_cluster && (long long)nitems * cs < 2LL * c->nsm) cs *= 2;
    int gat = 0, spcn = 0, cap = 0, pmax = 0;
    for (;;) {
        gat = spcn = cap = pmax = 0;
        for (const Item<real>& it : items) {
            const int P1 = it.ax[1].P, P0 = it.ax[0].P, Q1 = P1 / 2 + 1;
            const int lpc = (it.S[0] + cs - 1) / cs, cpc = (Q1 + cs - 1) / cs;
            gat = std::max(gat, it.S[0] * cpc);
            spcn = std::max(spcn, cpc * P0);
            cap = std::max(cap, std::max(lpc * P1, cpc * P0));
            pmax = std::max(pmax, std::max(P0, P1));
        }
        gat = (gat + 1) & ~1;   // keeps the spectrum rows that follow 16-byte aligned for the bulk copy
        const size_t need = sizeof(C) * (size_t)(gat + 2 * pmax + 2 * (cap + cap / 16 + 1)) +
                            sizeof(real) * (size_t)(spcn + 4);
        if (need <= budget) break;
        if (cs >= c->max_cluster) return KDEFFT_ERR_UNSUPPORTED;
        cs *= 2;
    }
    KCHK(sync_twiddles(c));
    const size_t bItems = sizeof(FusedItem<real>) * nitems;
    KCHK(staging_wait(c));
    KCHK(c->h_items.ensure(bItems));
    KCHK(c->items.ensure(bItems));
    KCHK(c->out.ensure(sizeof(double) * 2 * nitems));
    KCHK(c->h_out.ensure(sizeof(double) * 2 * nitems));
    {
        FusedItem<real>* fi = (FusedItem<real>*)c->h_items.p;
        for (int i = 0; i < nitems; ++i) {
            const Item<real>& it = items[i];
            FusedItem<real>& f = fi[i];
            std::memset(&f, 0, sizeof(f));
            f.S0 = it.S[0];
            f.S1 = it.S[1];
            f.off0 = it.off[0];
            f.off1 = it.off[1];
            f.nsig = it.nsig;
            f.delta0 = it.delta[0];
            f.delta1 = it.delta[1];
            for (int q = 0; q < MAXSIG; ++q) {
                f.lam[q][0] = it.lam[q][0];
                f.lam[q][1] = it.lam[q][1];
                f.lam[q][2] = it.lam[q][MAXD];
                f.lam[q][3] = it.lam[q][MAXD + 1];
                for (int e = 0; e < 4; ++e) f.laml[q][e] = (real)f.lam[q][e];
                f.nrm[q] = (real)it.nrm[q];
            }
            for (int h = 0; h < 2; ++h)
                for (int m = 0; m < it.nterm[h]; ++m) f.W[h][it.tsig[h][m]][it.the[h][m]] += it.tw8[h][m];
            f.a0 = it.ax[0];
            f.a1 = it.ax[1];
            f.spec = it.spec;
            f.scale = it.scale;
        }
    }
    double fl = 0.0, by = 0.0;
    for (const Item<real>& it : items) {
        const double P1 = it.ax[1].P, P0 = it.ax[0].P, Q1 = std::floor(P1 / 2) + 1;
        fl += it.S[0] * 5.0 * P1 * std::log2(P1) + Q1 * (5.0 * P0 * std::log2(P0) + 4.0 * P0);
        by += Q1 * P0 * sizeof(real);
    }
    const C* tw = (const C*)(sizeof(real) == 4 ? c->tw32.p : c->tw64.p);
    const std::vector<long long> sig = {2,
                                        (long long)sizeof(real),
                                        nitems,
                                        rmax,
                                        cs,
                                        gat,
                                        spcn,
                                        cap,
                                        pmax,
                                        (long long)(uintptr_t)c->items.p,
                                        (long long)(uintptr_t)c->h_items.p,
                                        (long long)(uintptr_t)tw,
                                        (long long)(uintptr_t)c->out.p,
                                        (long long)(uintptr_t)c->h_out.p};
    bool too_big = false;   // a 16-CTA cluster of this footprint does not fit the device
    auto issue = [&]() -> int {
        cudaEvent_t ev = prof_start(c);
        cudaError_t le = launch_fused2d<real>((const FusedItem<real>*)c->items.p, nitems, rmax, cs, gat, spcn, cap,
                                              pmax, tw, (double*)c->out.p, c->errflag, c->stream);
        if (le == cudaErrorNotSupported && cs > 8) {
            too_big = true;
            return KDEFFT_ERR_UNSUPPORTED;
        }
        KCU(le);
        prof_stop(c, ev, sizeof(real) == 4 ? "fused2d_f32" : "fused2d_f64", by, fl);
        KCU(cudaMemcpyAsync(c->h_out.p, c->out.p, sizeof(double) * 2 * nitems, cudaMemcpyDeviceToHost, c->stream));
        return KDEFFT_OK;
    };
    KCHK(staging_upload(c, c->items.p, bItems));
    const int ir = run_graph(c, sig, issue);
    if (too_big) {
        // stay at 8-CTA clusters from now on
        KCU(cudaStreamSynchronize(c->stream));
        c->staging_free = true;
        c->max_cluster = 8;
        return launch_fused<real>(c, items, out_host);
    }
    KCHK(ir);
    c->h2d += (int64_t)bItems;
    {
        HostTimer w(c, "host:wait");
        KCU(cudaStreamSynchronize(c->stream));
    }
    c->staging_free = true;
    c->d2h += (int64_t)(sizeof(double) * 2 * nitems);
    std::memcpy(out_host, c->h_out.p, sizeof(double) * 2 * nitems);
    prof_flush(c);
    KCHK(check_errflag(c));
    return KDEFFT_OK;
}

static std::vector<int> spectrum_key(const kdefft_ds ds, const int* P, size_t realsize) {
    std::vector<int> key(P, P + ds->d);
    key.push_back((int)realsize);
    return key;
}

// |F(c_zp)|^2 for every (dataset, P) in `need` that is not cached yet,
// computed in one batched launch sequence (split by the scratch budget)
template <typename real>
static int ensure_spectra(kdefft_ctx c, const std::vector<std::pair<kdefft_ds, std::array<int, 4>>>& need) {
    std::vector<Item<real>> items;
    std::vector<std::pair<kdefft_ds, std::vector<int>>> keys;
    std::vector<std::shared_ptr<DevBuf>> bufs;
    const long long budget = 1LL << 28;
    long long scratch = 0;
    auto flush = [&]() -> int {
        if (items.empty()) return KDEFFT_OK;
        // lines per tile: the default capacity, unless that leaves fewer than
        // two tiles per SM in the first pass (one small grid): then fewer
        // lines per tile, down to one line
        long long work = 0;   // complex elements of the first pass
        int pmax = 2;
        for (const Item<real>& it : items) {
            long long lines = 1;
            for (int k = 0; k < it.d - 1; ++k) lines *= it.S[k];
            work += lines * it.ax[it.d - 1].P;
            for (int k = 0; k < it.d; ++k) pmax = std::max(pmax, it.ax[k].P);
        }
        const int cap = (int)std::max<long long>(pmax, std::min<long long>(cap_elems(sizeof(real) == 8),
                                                                             work / (2LL * c->nsm)));
        PassLists pl;
        for (size_t i = 0; i < items.size(); ++i) tile_item(items[i], (int)i, cap, pl);
        KCHK(launch_items<real>(c, items, pl, items[0].d, nullptr));
        for (size_t i = 0; i < keys.size(); ++i) keys[i].first->spectra[keys[i].second] = bufs[i];
        items.clear();
        keys.clear();
        bufs.clear();
        scratch = 0;
        return KDEFFT_OK;
    };
    std::set<std::pair<kdefft_ds, std::vector<int>>> queued;
    for (const auto& np : need) {
        kdefft_ds ds = np.first;
        const int* P = np.second.data();
        std::vector<int> key = spectrum_key(ds, P, sizeof(real));
        if (ds->spectra.count(key) || queued.count({ds, key})) continue;
        queued.insert({ds, key});
        auto buf = std::make_shared<DevBuf>(&c->cache);
        KCHK(buf->ensure(sizeof(real) * spec_elems(ds->d, P)));
        Item<real> item;
        std::memset(&item, 0, sizeof(item));
        item.d = ds->d;
        item.kind = 1;
        KCHK(fill_axes(c, ds->d, P, item));
        for (int k = 0; k < ds->d; ++k) {
            item.S[k] = (int)ds->M[k];
            item.off[k] = 0;
        }
        const bool ds64 = ds->opts.precision == KDEFFT_FP64;
        if (sizeof(real) == 8 && !ds64) {
            // FP64 work on an FP32 dataset: widen the counts once
            if (!ds->counts64.p) {
                KCHK(ds->counts64.ensure(sizeof(double) * (size_t)ds->ncells));
                c->launches++;
                KCU(launch_f32_to_f64((const float*)ds->counts.p, (double*)ds->counts64.p, ds->ncells, c->stream));
            }
            item.counts = (const real*)ds->counts64.p;
        } else {
            item.counts = (const real*)ds->counts.p;
        }
        item.spec_out = (real*)buf->p;
        const long long sn = scratch_need(item);
        if (!items.empty() && scratch + sn > budget) KCHK(flush());
        scratch += sn;
        items.push_back(item);
        keys.push_back({ds, key});
        bufs.push_back(buf);
    }
    return flush();
}

// Evaluate every grid of rs (value = Eq. 25 for that lag kernel).
// ============================================================ lag-domain engine
static long long pmin_smooth(long long m) { return next_smooth(m); }

// a_j = sum_i c_i c_{i+j} on the half box A (j_0 in [0, A_0], |j_k| <= A_k),
// layout [j_{d-1}]..[j_0], from the FP64 count spectrum at P_k >= M_k + A_k
// (no aliasing on the box) by separable pruned inverse DFTs in FP64; the
// last pass also writes the FP32 copy.  A box grows (by half of itself at
// least) when a request needs more.  Every dataset of `req` is brought up to
// date with one batched spectrum launch sequence and stream-ordered passes
// through context buffers (no synchronisation).
// lines per CTA of an autocorrelation pass of length P over `lines` lines:
// as many as fit 96 KB of shared memory (two resident CTAs per SM), but no
// more than leave two CTAs per SM busy; at least one
static int acorr_lines(int P, long long lines, int nsm) {
    int nl = 1;
    while (nl < 64 && acorr_smem_bytes(P, nl + 1) <= (size_t)96 * 1024) ++nl;
    const long long spread = std::max<long long>(1, lines / (2LL * nsm));
    return (int)std::min<long long>(nl, spread);
}

// Cache key of a count spectrum held as FP32 pairs (the autocorrelation input
// of FP32 datasets): element size 8 as for FP64, told apart by this tag.
static constexpr size_t kPairTag = 9;
// Largest radix of the FP32-pair transforms.  A pair butterfly is a long
// chain of dependent FP32 operations, so small radices (more threads busy
// per stage, shorter chains) win: measured for the count spectrum and
// autocorrelation of a 256^2 grid at P = 384 (n = 1e5), 42 µs with radices up
// to 5, 55 µs up to 8, 84 µs up to 16 (the FP64 passes: 81 µs); 128^3 at
// P = 180 (n = 1e6): 405, 406, 494 µs (FP64: 921 µs).
static constexpr int kPairRadix = 5;

// |F(c_zp)|^2 at padded P for FP32 datasets, in FP32-pair arithmetic: d
// forward passes of k_spec_df per dataset, one launch per pass level for
// every dataset of a dimension.  The first level transforms the last axis
// of the FP32 counts (half spectrum), the middle levels the interior axes,
// the last level axis 0 and writes |X|^2 in the spectrum layout
// [w_{d-1}]..[w_1][w_0] that the autocorrelation passes read.  Intermediate
// lines go through the context's two pass buffers (stream-ordered reuse).
// The launches of a batch of FP32-pair count-spectrum passes, whose job table
// is already on its way to the device: issued by the caller (in one graph
// with the autocorrelation passes that read the spectra).
struct SpecLaunches {
    SpecJob* jd = nullptr;
    size_t table_bytes = 0;   // the job table, in h_specjobs until the caller's copy
    struct L {
        size_t slot;
        int n;
        long long blocks;
        size_t sm;
    };
    std::vector<L> lv;
    double by = 0.0, fl = 0.0;
};

static int ensure_spectra_df(kdefft_ctx c, const std::vector<std::pair<kdefft_ds, std::array<int, 4>>>& need,
                             SpecLaunches& sl) {
    struct Sj {
        kdefft_ds ds;
        std::array<int, 4> P;
        std::vector<int> key;
        std::shared_ptr<DevBuf> buf;
        long long E[MAXD];   // frequencies kept per axis: P_k, the half spectrum on the last axis
        size_t off, most;
    };
    std::vector<Sj> todo;
    std::set<std::pair<kdefft_ds, std::vector<int>>> queued;
    for (const auto& np : need) {
        kdefft_ds ds = np.first;
        std::vector<int> key = spectrum_key(ds, np.second.data(), kPairTag);
        if (ds->spectra.count(key) || queued.count({ds, key})) continue;
        queued.insert({ds, key});
        Sj j{ds, np.second, key, std::make_shared<DevBuf>(&c->cache), {0, 0, 0, 0}, 0, 0};
        KCHK(j.buf->ensure(sizeof(double) * spec_elems(ds->d, np.second.data())));
        todo.push_back(std::move(j));
    }
    if (todo.empty()) return KDEFFT_OK;
    size_t pool = 0;
    for (Sj& j : todo) {
        const int d = j.ds->d;
        for (int k = 0; k < d; ++k) {
            j.E[k] = (k == d - 1) ? j.P[k] / 2 + 1 : j.P[k];
            twiddle_offset(c, j.P[k]);
        }
        // the largest intermediate: after the pass on axis k (k >= 1), the
        // untransformed axes m < k hold M_m values and the others E_m
        j.most = 0;
        for (int k = d - 1; k >= 1; --k) {
            long long e = 1;
            for (int m = 0; m < d; ++m) e *= (m < k) ? j.ds->M[m] : j.E[m];
            j.most = std::max(j.most, (size_t)e);
        }
        j.off = pool;
        pool += (j.most + 1) & ~(size_t)1;
    }
    KCHK(sync_twiddles(c));
    KCHK(c->acbuf[0].ensure(sizeof(double2) * std::max<size_t>(pool, 1)));
    KCHK(c->acbuf[1].ensure(sizeof(double2) * std::max<size_t>(pool, 1)));
    double2* pools[2] = {(double2*)c->acbuf[0].p, (double2*)c->acbuf[1].p};
    std::vector<SpecJob> all;
    std::vector<SpecLaunches::L>& lv = sl.lv;
    double& fl = sl.fl;
    double& by = sl.by;
    for (int dim = 1; dim <= MAXD; ++dim) {
        std::vector<size_t> sel;
        for (size_t u = 0; u < todo.size(); ++u)
            if (todo[u].ds->d == dim) sel.push_back(u);
        if (sel.empty()) continue;
        for (int lev = 0; lev < dim; ++lev) {
            const int k = dim - 1 - lev;   // the axis of this level
            const size_t slot = all.size();
            all.resize(slot + sel.size());
            for (size_t v = 0; v < sel.size(); ++v) {
                const Sj& j = todo[sel[v]];
                kdefft_ds ds = j.ds;
                SpecJob& a = all[slot + v];
                std::memset(&a, 0, sizeof(a));
                a.d = dim;
                a.in_f = (lev == 0) ? (const float*)ds->counts.p : nullptr;
                a.in_c = (lev == 0) ? nullptr : (const void*)(pools[(lev - 1) & 1] + j.off);
                long long O = 1, I = 1;
                for (int m = 0; m < k; ++m) O *= ds->M[m];
                for (int m = k + 1; m < dim; ++m) I *= j.E[m];
                a.O = O;
                a.I = I;
                a.X = (int)ds->M[k];
                a.Y = (int)j.E[k];
                if (k == 0) {
                    a.out_s = j.buf->p;
                    for (int m = 1; m < dim; ++m) a.ext[m] = (int)j.E[m];
                } else {
                    a.out_c = (void*)(pools[lev & 1] + j.off);
                }
                a.ap.tw_off = twiddle_offset(c, j.P[k]);
                if (!radix_plan(j.P[k], a.ap, kPairRadix)) return fail(KDEFFT_ERR_UNSUPPORTED, "no radix plan for P");
                a.nl = acorr_lines(j.P[k], O * I, c->nsm);
                fl += 5.0 * j.P[k] * std::log2((double)j.P[k]) * (double)(O * I);
                by += (lev == 0 ? 4.0 : 16.0) * (double)(O * I) * a.X + (k == 0 ? 8.0 : 16.0) * (double)(O * I) * a.Y;
            }
            SpecLaunches::L L{slot, (int)sel.size(), 0, 0};
            KCU(spec_plan(all.data() + slot, L.n, &L.blocks, &L.sm));
            lv.push_back(L);
        }
    }
    KCHK(c->specjobs.ensure(sizeof(SpecJob) * all.size()));
    if (!c->specjobs_free) KCU(cudaEventSynchronize(c->specjobs_ev));
    KCHK(c->h_specjobs.ensure(sizeof(SpecJob) * all.size()));
    std::memcpy(c->h_specjobs.p, all.data(), sizeof(SpecJob) * all.size());
    sl.jd = (SpecJob*)c->specjobs.p;
    sl.table_bytes = sizeof(SpecJob) * all.size();
    // the spectra are registered now; the caller copies the table up and
    // issues the passes before any launch that reads them
    for (Sj& j : todo) j.ds->spectra[j.key] = j.buf;
    return KDEFFT_OK;
}

// Work that follows the autocorrelation passes on the stream (the device
// search): its launch signature and its copies and launches.
struct StreamTail {
    // called once the autocorrelation boxes and buffers are final: sets up
    // the work's parameters and appends its launch signature
    std::function<int(std::vector<long long>&)> prepare;
    std::function<int()> issue;
};

// Grow the count autocorrelation of each dataset to the half box it needs
// (the FP32-pair or FP64 count spectrum first).  With a tail, the tail's work
// joins the same launch sequence (one graph replay for all of it); it runs on
// its own when there is nothing to grow.
static int ensure_autocorr_many(kdefft_ctx c, const std::vector<std::pair<kdefft_ds, std::array<int, 4>>>& req,
                                StreamTail* tail = nullptr) {
    HostTimer ht(c, "host:acorr");
    struct Job {
        kdefft_ds ds;
        int A[4], P[4];
    };
    std::vector<Job> jobs;
    std::vector<std::pair<kdefft_ds, std::array<int, 4>>> specs, specs_df;
    for (const auto& rq : req) {
        kdefft_ds ds = rq.first;
        const int d = ds->d;
        bool covered = ds->acA[0] >= 0;
        for (int k = 0; k < d; ++k) covered = covered && ds->acA[k] >= rq.second[k];
        if (covered) continue;
        Job jb{ds, {0, 0, 0, 0}, {1, 1, 1, 1}};
        for (int k = 0; k < d; ++k) {
            const int grow = ds->acA[k] >= 0 ? ds->acA[k] + ds->acA[k] / 2 : 0;
            jb.A[k] = (int)std::min<long long>(ds->M[k] - 1, std::max(rq.second[k], grow));
            jb.P[k] = (int)pmin_smooth(ds->M[k] + jb.A[k]);
            if (jb.P[k] > MAXP) return KDEFFT_ERR_UNSUPPORTED;
        }
        jobs.push_back(jb);
        (ds->opts.precision == KDEFFT_FP64 ? specs : specs_df).push_back({ds, {jb.P[0], jb.P[1], jb.P[2], jb.P[3]}});
    }
    // FP64 datasets: the FP64 transforms; FP32 datasets: FP32 pairs (about 44
    // bits, on the FP32 pipes), far beyond their FP32 counts' own rounding
    if (!specs.empty()) KCHK(ensure_spectra<double>(c, specs));
    SpecLaunches sl;
    if (!specs_df.empty()) KCHK(ensure_spectra_df(c, specs_df, sl));
    for (const Job& jb : jobs)
        for (int k = 0; k < jb.ds->d; ++k) twiddle_offset(c, jb.P[k]);
    KCHK(sync_twiddles(c));
    const double2* tw = (const double2*)c->tw64.p;
    // Per dataset, the sizes of its passes; pass buffers at offsets in the
    // two context pools; then every pass level is one launch over all
    // datasets of that dimension (level k transforms axis k: [w_{d-1} ..
    // w_{k+1}][w_k][j_{k-1} .. j_0] -> [..][j_k][..]; the last level is the
    // half-spectrum axis, written as real FP64 and FP32).
    struct Plan {
        const double* S;
        long long O0;      // rows of the innermost pass
        size_t most;       // complex elements of the largest intermediate
        size_t off;        // offset in the pools
        double ptot;
        int Q;
    };
    std::vector<Plan> plan(jobs.size());
    size_t pool = 0;
    double fl = 0.0, by = 0.0;
    for (size_t u = 0; u < jobs.size(); ++u) {
        const Job& jb = jobs[u];
        kdefft_ds ds = jb.ds;
        const int d = ds->d;
        const int* A = jb.A;
        const int* P = jb.P;
        const bool pairs = ds->opts.precision != KDEFFT_FP64;
        auto sit = ds->spectra.find(spectrum_key(ds, P, pairs ? kPairTag : sizeof(double)));
        if (sit == ds->spectra.end()) return fail(KDEFFT_ERR_CUDA, "count spectrum missing");
        Plan& pl = plan[u];
        pl.S = (const double*)sit->second->p;
        pl.Q = P[d - 1] / 2 + 1;
        pl.ptot = 1.0;
        long long nbox = 1;
        for (int k = 0; k < d; ++k) {
            nbox *= (k == 0) ? (A[0] + 1) : (2 * A[k] + 1);
            pl.ptot *= P[k];
        }
        KCHK(ds->ac64.ensure(sizeof(double) * nbox));
        KCHK(ds->ac32.ensure(sizeof(float) * nbox));
        pl.O0 = pl.Q;
        for (int k = 1; k <= d - 2; ++k) pl.O0 *= P[k];
        pl.most = 0;
        {
            // a length-P complex transform per line: 5 P log2 P flops
            long long o = pl.O0, ii = 1;
            for (int k = 0; k < d - 1; ++k) {
                const int J = (k == 0) ? A[0] + 1 : 2 * A[k] + 1;
                pl.most = std::max(pl.most, (size_t)(o * J * ii));
                fl += 5.0 * P[k] * std::log2((double)P[k]) * (double)(o * ii);
                ii *= J;
                if (k + 1 <= d - 2) o /= P[k + 1];
            }
            fl += 5.0 * P[d - 1] * std::log2((double)P[d - 1]) * (double)ii;
        }
        pl.off = pool;
        pool += (pl.most + 1) & ~(size_t)1;
        double b = 8.0 * pl.Q;
        for (int k = 0; k < d - 1; ++k) b *= P[k];
        by += b;
    }
    if (!jobs.empty()) {
        KCHK(c->acbuf[0].ensure(sizeof(double2) * std::max<size_t>(pool, 1)));
        KCHK(c->acbuf[1].ensure(sizeof(double2) * std::max<size_t>(pool, 1)));
        // one table slice per launch (at most MAXD launches per dataset); all
        // slices go up in one copy from pinned memory, so that the host does
        // not wait for the stream (a pageable copy would)
        KCHK(c->acjobs.ensure(sizeof(AcorrJob) * jobs.size() * MAXD));
        AcorrJob* jd = (AcorrJob*)c->acjobs.p;
        double2* pool0 = (double2*)c->acbuf[0].p;
        double2* pool1 = (double2*)c->acbuf[1].p;
        std::vector<AcorrJob> all;
        struct Launch {
            size_t slot;
            int n;
            long long blocks;
            size_t sm;
            bool pairs;   // FP32-pair passes (FP32 datasets)
        };
        std::vector<Launch> lv;
        for (int pr = 0; pr < 2; ++pr)
        for (int dim = 1; dim <= MAXD; ++dim) {
            std::vector<size_t> sel;
            for (size_t u = 0; u < jobs.size(); ++u)
                if (jobs[u].ds->d == dim && (jobs[u].ds->opts.precision != KDEFFT_FP64) == (pr == 1)) sel.push_back(u);
            if (sel.empty()) continue;
            // level k of every selected dataset
            std::vector<long long> O(sel.size()), I(sel.size(), 1);
            for (size_t v = 0; v < sel.size(); ++v) O[v] = plan[sel[v]].O0;
            for (int k = 0; k < dim; ++k) {
                const bool last = (k == dim - 1);
                const size_t slot = all.size();
                all.resize(slot + sel.size());
                for (size_t v = 0; v < sel.size(); ++v) {
                    const Job& jb = jobs[sel[v]];
                    const Plan& pl = plan[sel[v]];
                    AcorrJob& a = all[slot + v];
                    std::memset(&a, 0, sizeof(a));
                    // ping-pong: level k reads pool (k+1)&1, writes pool k&1
                    double2* rd = ((k & 1) ? pool0 : pool1) + pl.off;
                    double2* wr = ((k & 1) ? pool1 : pool0) + pl.off;
                    a.in_r = (k == 0) ? pl.S : nullptr;
                    a.in_c = (k == 0) ? nullptr : rd;
                    a.O = last ? 1 : O[v];
                    a.I = I[v];
                    a.W = last ? pl.Q : jb.P[k];
                    a.J = (k == 0) ? jb.A[0] + 1 : 2 * jb.A[k] + 1;
                    a.jlo = (k == 0) ? 0 : -jb.A[k];
                    a.ap.tw_off = twiddle_offset(c, jb.P[k]);
                    if (!radix_plan(jb.P[k], a.ap, pr == 1 ? kPairRadix : 16))
                        return fail(KDEFFT_ERR_UNSUPPORTED, "no radix plan for P");
                    a.nl = acorr_lines(jb.P[k], a.O * a.I, c->nsm);
                    a.half = last ? 1 : 0;
                    a.scale = last ? 1.0 / pl.ptot : 1.0;
                    if (last) {
                        a.out_r = (double*)jb.ds->ac64.p;
                        a.out_r32 = (float*)jb.ds->ac32.p;
                    } else {
                        a.out_c = wr;
                    }
                }
                Launch L{slot, (int)sel.size(), 0, 0, pr == 1};
                KCU(acorr_plan(all.data() + slot, L.n, &L.blocks, &L.sm));
                lv.push_back(L);
                for (size_t v = 0; v < sel.size(); ++v) {
                    const Job& jb = jobs[sel[v]];
                    const int J = (k == 0) ? jb.A[0] + 1 : 2 * jb.A[k] + 1;
                    I[v] *= J;
                    if (k + 1 <= dim - 2) O[v] /= jb.P[k + 1];
                }
            }
        }
        for (const Job& jb : jobs)
            for (int k = 0; k < 4; ++k) jb.ds->acA[k] = (k < jb.ds->d) ? jb.A[k] : 0;
        if (!c->acjobs_free) KCU(cudaEventSynchronize(c->acjobs_ev));
        const size_t acb = sizeof(AcorrJob) * all.size();
        KCHK(c->h_acjobs.ensure(acb));
        std::memcpy(c->h_acjobs.p, all.data(), acb);
        // the table copies, the count-spectrum passes (FP32 datasets), the
        // autocorrelation passes and the tail in one launch sequence,
        // replayed as a CUDA graph when its tables, sizes and launch shapes
        // repeat (the copies read the pinned tables when the graph runs)
        std::vector<long long> sig = {7, (long long)(uintptr_t)sl.jd, (long long)(uintptr_t)jd,
                                      (long long)(uintptr_t)c->h_specjobs.p, (long long)sl.table_bytes,
                                      (long long)(uintptr_t)c->h_acjobs.p, (long long)acb,
                                      (long long)(uintptr_t)c->twdf.p, (long long)(uintptr_t)tw,
                                      (long long)sl.lv.size()};
        for (const auto& L : sl.lv) sig.insert(sig.end(), {(long long)L.slot, L.n, L.blocks, (long long)L.sm});
        for (const Launch& L : lv)
            sig.insert(sig.end(), {(long long)L.slot, L.n, L.blocks, (long long)L.sm, L.pairs ? 1 : 0});
        if (tail) KCHK(tail->prepare(sig));
        auto issue = [&]() -> int {
            if (sl.table_bytes)
                KCU(cudaMemcpyAsync(sl.jd, c->h_specjobs.p, sl.table_bytes, cudaMemcpyHostToDevice, c->stream));
            KCU(cudaMemcpyAsync(jd, c->h_acjobs.p, acb, cudaMemcpyHostToDevice, c->stream));
            if (!sl.lv.empty()) {
                cudaEvent_t es = prof_start(c);
                c->launches--;   // counted per launch below
                for (const auto& L : sl.lv) {
                    c->launches++;
                    KCU(launch_spec_df(sl.jd + L.slot, L.n, L.blocks, L.sm, c->twdf.p, c->stream));
                }
                prof_stop(c, es, "spec_df", sl.by, sl.fl);
            }
            cudaEvent_t ev = prof_start(c);
            c->launches--;   // counted per launch below
            for (const Launch& L : lv) {
                c->launches++;
                if (L.pairs)
                    KCU(launch_acorr_df(jd + L.slot, L.n, L.blocks, L.sm, c->twdf.p, c->stream));
                else
                    KCU(launch_acorr(jd + L.slot, L.n, L.blocks, L.sm, tw, c->stream));
            }
            prof_stop(c, ev, "acorr", by, fl);
            if (tail) KCHK(tail->issue());
            return KDEFFT_OK;
        };
        KCHK(run_graph(c, sig, issue));
        // the pinned tables are free again once this work has run
        if (sl.table_bytes) {
            KCU(cudaEventRecord(c->specjobs_ev, c->stream));
            c->specjobs_free = false;
        }
        KCU(cudaEventRecord(c->acjobs_ev, c->stream));
        c->acjobs_free = false;
        c->h2d += (int64_t)(sl.table_bytes + acb);
        tail = nullptr;
    }
    if (tail) {
        std::vector<long long> sig = {9};
        KCHK(tail->prepare(sig));
        KCHK(run_graph(c, sig, tail->issue));
    }
    return KDEFFT_OK;
}

// highest derivative order among the terms of a grid pair
static int pair_order(const ReqSet& rs, const std::pair<int, int>& pr, int d) {
    int R = 0;
    for (int gi : {pr.first, pr.second}) {
        if (gi < 0) continue;
        for (const Term& t : rs.grids[gi].terms) {
            int o = 0;
            for (int k = 0; k < d; ++k) o += t.alpha[k];
            R = std::max(R, o);
        }
    }
    return R;
}

// the lag-domain engine computes exactly the FFT route's value when the
// padding has no aliasing (P_k >= M_k + L_k on every axis)
template <typename real>
static bool lag_eligible(kdefft_ctx c, const ReqSet& rs, const std::pair<int, int>& pr) {
    if (!c->lag) return false;
    const GridReq& g = rs.grids[pr.first];
    const int d = g.ds->d;
    long long pts = g.L[0] + 1;   // half-box points: the lag kernel indexes them in 32 bits
    for (int k = 0; k < d; ++k) {
        if (g.P[k] < g.ds->M[k] + g.L[k]) return false;
        if (k > 0) pts *= 2 * g.L[k] + 1;
    }
    if (pts > (1LL << 32)) return false;
    return lag_table_size(d, pair_order(rs, pr, d), sizeof(real) == 8) > 0;
}

// Granlund and Montgomery's unsigned division by an invariant integer
// 1 <= v < 2^32 for 32-bit numerators ("Division by invariant integers
// using multiplication", 1994): with l = ceil(log2 v), the multiplier
// m = floor(2^32 (2^l - v) / v) + 1 and the shifts s1 = min(l, 1),
// s2 = max(l - 1, 0) give floor(n / v) = (t + ((n - t) >> s1)) >> s2,
// t = mulhi(m, n).  sh packs s1 | s2 << 8.
static void invariant_div(uint32_t v, unsigned int& m, int& sh) {
    int l = 0;
    while ((1ULL << l) < v) ++l;
    m = (unsigned int)(((((1ULL << l) - v) << 32) / v) + 1);
    sh = std::min(l, 1) | (std::max(l - 1, 0) << 8);
}

// The lag-domain work of one precision in a run, built on the host: the
// items (LagItem<real>), their tiles and dense weights, the derivative-order
// classes (R, first tile, tiles; one launch each) and the grid pairs in item
// order.  run_lag builds it; issue_lag uploads and launches the batches of
// both precisions of a run together.
struct LagBatch {
    bool dbl = false;
    int d = 0;
    int nitems = 0;
    std::vector<LagItem<float>> it32;    // the items (it64 for FP64)
    std::vector<LagItem<double>> it64;
    std::vector<float> w32;              // the dense weights (w64 for FP64)
    std::vector<double> w64;
    std::vector<LagTile> tiles;
    std::vector<std::array<int, 3>> classes;
    std::vector<std::pair<int, int>> pairs;
    double fl = 0.0, by = 0.0;   // algorithmic flops and bytes of the batch
    template <typename real>
    std::vector<LagItem<real>>& items() {
        if constexpr (sizeof(real) == 8) return it64; else return it32;
    }
    template <typename real>
    std::vector<real>& wpool() {
        if constexpr (sizeof(real) == 8) return w64; else return w32;
    }
    const void* item_bytes() const { return dbl ? (const void*)it64.data() : (const void*)it32.data(); }
    size_t item_size() const { return dbl ? sizeof(LagItem<double>) * it64.size() : sizeof(LagItem<float>) * it32.size(); }
    const void* w_bytes() const { return dbl ? (const void*)w64.data() : (const void*)w32.data(); }
    size_t w_size() const { return dbl ? sizeof(double) * w64.size() : sizeof(float) * w32.size(); }
};

// Build the lag-domain batch for the grid pairs (the count autocorrelation
// box they need is grown first).  (Building a large set in chunks, each
// issued while the next is built, was measured slower: each chunk's launch
// leaves the GPU partly idle at its tail.)

template <typename real>
static int run_lag(kdefft_ctx c, ReqSet& rs, std::vector<std::pair<int, int>> pairs, std::vector<LagBatch>& out) {
    if (pairs.empty()) return KDEFFT_OK;
    const bool dbl = sizeof(real) == 8;
    const int d = rs.grids[pairs[0].first].ds->d;
    {
        std::map<kdefft_ds, std::array<int, 4>> need;
        for (const auto& pr : pairs) {
            const GridReq& g = rs.grids[pr.first];
            auto& a = need[g.ds];
            for (int k = 0; k < d; ++k) a[k] = std::max(a[k], g.L[k]);
        }
        std::vector<std::pair<kdefft_ds, std::array<int, 4>>> rq(need.begin(), need.end());
        KCHK(ensure_autocorr_many(c, rq));
    }
    HostTimer hbuild(c, "host:lag_build");
    // order classes, contiguous
    std::vector<int> Re(pairs.size());
    for (size_t i = 0; i < pairs.size(); ++i) Re[i] = (pair_order(rs, pairs[i], d) + 1) & ~1;
    std::vector<size_t> ord(pairs.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return Re[a] < Re[b]; });
    HermiteIndex& hx = hindex();
    // fixed tiles, so that an item's sum depends on the item alone, not on
    // the batch it came in: 4096 points in FP32 (smaller tiles halved the
    // throughput of batches: per-tile work is then too small for a CTA), 256
    // in FP64 (the points are slow on the FP64 pipe: more CTAs in flight, one
    // point per thread)
    const long long T = dbl ? 32 * kLagSlices : 4096;
    const size_t ni = ord.size();
    LagBatch bt;
    bt.dbl = dbl;
    bt.d = d;
    std::vector<LagItem<real>>& items = bt.items<real>();
    std::vector<real>& wpool = bt.wpool<real>();
    // layout (serial): each item's tiles and weights at fixed offsets, the
    // order classes, the algorithmic work
    std::vector<long long> tile0(ni + 1), woff(ni + 1), npts(ni);
    tile0[0] = 0;
    woff[0] = 0;
    for (size_t q = 0; q < ni; ++q) {
        const size_t u = ord[q];
        const GridReq& g = rs.grids[pairs[u].first];
        const int nsig = rs.specs[g.spec].nsig;
        long long pts = g.L[0] + 1;
        for (int k = 1; k < d; ++k) pts *= 2 * g.L[k] + 1;
        npts[q] = pts;
        const int N = lag_table_size(d, Re[u], dbl);
        tile0[q + 1] = tile0[q] + (pts + T - 1) / T;
        woff[q + 1] = woff[q] + 2LL * nsig * N;
        if (bt.classes.empty() || bt.classes.back()[0] != Re[u]) bt.classes.push_back({Re[u], (int)tile0[q], 0});
        bt.classes.back()[2] += (int)(tile0[q + 1] - tile0[q]);
        bt.fl += (double)pts * nsig * (2.0 * d * d + 8.0 * N);
        bt.by += (double)pts * sizeof(real);
        bt.pairs.push_back(pairs[u]);
    }
    if (tile0[ni] > 0x7fffffffLL || woff[ni] > 0x7fffffffLL)
        return fail(KDEFFT_ERR_UNSUPPORTED, "lag batch too large");
    items.resize(ni);
    bt.tiles.resize((size_t)tile0[ni]);
    wpool.assign((size_t)woff[ni], real(0));
    // inverse covariances and normalisations once per kernel spec (the pairs
    // of one bandwidth share them), then the items: both over index ranges
    // that may run on several host threads (each writes its own entries;
    // the result does not depend on the split)
    struct SpecInv {
        double lam[MAXSIG][MAXD * MAXD];
        double nrm[MAXSIG];
    };
    std::vector<char> used(rs.specs.size(), 0);
    for (size_t q = 0; q < ni; ++q) used[rs.grids[pairs[ord[q]].first].spec] = 1;
    std::vector<SpecInv> sinv(rs.specs.size());
    std::atomic<int> err{KDEFFT_OK};
    host_parallel_for(rs.specs.size(), 2048, [&](size_t s0, size_t s1) {
        for (size_t si = s0; si < s1; ++si) {
            if (!used[si]) continue;
            const KSpec& sp = rs.specs[si];
            for (int s = 0; s < sp.nsig; ++s) {
                Mat inv;
                double det;
                if (!spd_inv_det(sp.sig[s], inv, det)) {
                    err = KDEFFT_ERR_NOT_SPD;
                    return;
                }
                for (int a = 0; a < d; ++a)
                    for (int b = 0; b < d; ++b) sinv[si].lam[s][a * MAXD + b] = inv(a, b);
                sinv[si].nrm[s] = std::pow(2.0 * M_PI, -0.5 * d) / std::sqrt(det);
            }
        }
    });
    if (err != KDEFFT_OK) return fail(KDEFFT_ERR_NOT_SPD, "a kernel covariance is not positive definite");
    host_parallel_for(ni, 2048, [&](size_t q0, size_t q1) {
        for (size_t q = q0; q < q1; ++q) {
            const size_t u = ord[q];
            const auto& pr = pairs[u];
            const GridReq& g = rs.grids[pr.first];
            const KSpec& sp = rs.specs[g.spec];
            kdefft_ds ds = g.ds;
            LagItem<real>& it = items[q];
            std::memset(&it, 0, sizeof(it));
            it.d = d;
            it.nsig = sp.nsig;
            it.R = Re[u];
            for (int k = 0; k < d; ++k) {
                it.L[k] = g.L[k];
                it.A[k] = ds->acA[k];
                it.delta[k] = (real)ds->delta[k];
                invariant_div((uint32_t)(k == 0 ? g.L[0] + 1 : 2 * g.L[k] + 1), it.qm[k], it.qs[k]);
            }
            const SpecInv& si = sinv[g.spec];
            for (int s = 0; s < sp.nsig; ++s) {
                for (int a = 0; a < d; ++a)
                    for (int b = 0; b < d; ++b) it.lam[s][a * MAXD + b] = (real)si.lam[s][a * MAXD + b];
                it.nrm[s] = (real)si.nrm[s];
            }
            it.acorr = dbl ? (const real*)ds->ac64.p : (const real*)ds->ac32.p;
            const int N = lag_table_size(d, it.R, dbl);
            it.w_off = (int)woff[q];
            const int gi[2] = {pr.first, pr.second};
            for (int h = 0; h < 2; ++h) {
                if (gi[h] < 0) continue;
                for (const Term& t : rs.grids[gi[h]].terms) {
                    int o = 0;
                    for (int k = 0; k < d; ++k) o += t.alpha[k];
                    const int hidx = hx.idx(d, t.alpha);
                    if (hidx < 0 || hidx >= N) {
                        err = KDEFFT_ERR_UNSUPPORTED;
                        return;
                    }
                    wpool[it.w_off + (h * sp.nsig + t.sig) * N + hidx] += (real)(((o & 1) ? -1.0 : 1.0) * t.w);
                }
            }
            const double nn = (double)ds->n;
            it.scale = 1.0 / (nn * nn);
            it.tile0 = (int)tile0[q];
            it.ntile = (int)(tile0[q + 1] - tile0[q]);
            const long long pts = npts[q];
            long long f = 0;
            for (long long tq = tile0[q]; tq < tile0[q + 1]; ++tq, f += T)
                bt.tiles[tq] = LagTile{(int)q, (int)std::min(T, pts - f), f};
        }
    });
    if (err != KDEFFT_OK) return fail(KDEFFT_ERR_UNSUPPORTED, "derivative order too high");
    bt.nitems = (int)items.size();
    out.push_back(std::move(bt));
    return KDEFFT_OK;
}

// Upload the lag batches of a run in one copy and launch them (one tiled
// launch per batch and derivative-order class, then one fixed-order sum of
// every item's tile partials), then one copy of all values back; the values
// are read by flush_reads.
static int issue_lag(kdefft_ctx c, ReqSet& rs, std::vector<LagBatch>& bts) {
    if (bts.empty()) return KDEFFT_OK;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    struct Lay {
        size_t oI, oT, oW;
        int item0;
        long long tile0;   // first partial pair of the batch
    };
    std::vector<Lay> lay(bts.size());
    size_t bytes = 0;
    int nit = 0;
    long long ntl = 0;   // partial pairs of the run
    std::vector<LagSum> sums;
    for (size_t b = 0; b < bts.size(); ++b) {
        const LagBatch& bt = bts[b];
        lay[b].oI = bytes;
        bytes += al(bt.item_size());
        lay[b].oT = bytes;
        bytes += al(sizeof(LagTile) * bt.tiles.size());
        lay[b].oW = bytes;
        bytes += al(std::max<size_t>(bt.w_size(), 16));
        lay[b].item0 = nit;
        lay[b].tile0 = ntl;
        const int ps = bt.dbl ? kLagSlices : 1;   // partial pairs per tile
        for (int i = 0; i < bt.nitems; ++i) {
            // the item's tile range and scale, wherever its precision keeps them
            int t0i, nti;
            double sc;
            if (bt.dbl) {
                const LagItem<double>& q = bt.it64[i];
                t0i = q.tile0, nti = q.ntile, sc = q.scale;
            } else {
                const LagItem<float>& q = bt.it32[i];
                t0i = q.tile0, nti = q.ntile, sc = q.scale;
            }
            sums.push_back(LagSum{ntl + (long long)t0i * ps, nti, ps, sc});
        }
        nit += bt.nitems;
        ntl += (long long)bt.tiles.size() * ps;
    }
    const size_t oS = bytes;
    bytes += al(sizeof(LagSum) * sums.size());
    KCHK(staging_wait(c));
    KCHK(c->h_items.ensure(bytes));
    KCHK(c->items.ensure(bytes));
    KCHK(c->partial.ensure(sizeof(double) * 2 * (size_t)ntl));
    KCHK(c->out.ensure(sizeof(double) * 2 * (size_t)nit));
    // results go behind those of earlier lag launches still on their way
    const size_t need = 2 * (size_t)nit;
    if (c->h_out.cap < sizeof(double) * (c->hout_used + need)) {
        // (the results still on their way point into h_out: read them first;
        // grow by at least 4x, so that the next chunks of a large run fit)
        const size_t grow = std::max(need, 4 * (c->h_out.cap / sizeof(double)));
        KCHK(flush_reads(c));
        KCHK(c->h_out.ensure(sizeof(double) * grow));
    }
    const size_t off = c->hout_used;
    unsigned char* h = (unsigned char*)c->h_items.p;
    unsigned char* dbase = (unsigned char*)c->items.p;
    double* part = (double*)c->partial.p;
    double* dout = (double*)c->out.p;
    std::memcpy(h + oS, sums.data(), sizeof(LagSum) * sums.size());
    std::vector<long long> sig = {3, (long long)(uintptr_t)dbase, (long long)(uintptr_t)h, (long long)bytes,
                                  (long long)(uintptr_t)part, (long long)(uintptr_t)dout, (long long)oS, nit,
                                  (long long)(uintptr_t)c->h_out.p, (long long)off};
    for (size_t b = 0; b < bts.size(); ++b) {
        const LagBatch& bt = bts[b];
        std::memcpy(h + lay[b].oI, bt.item_bytes(), bt.item_size());
        std::memcpy(h + lay[b].oT, bt.tiles.data(), sizeof(LagTile) * bt.tiles.size());
        if (bt.w_size()) std::memcpy(h + lay[b].oW, bt.w_bytes(), bt.w_size());
        sig.insert(sig.end(), {bt.dbl ? 8 : 4, bt.d, bt.nitems, (long long)bt.tiles.size(), (long long)lay[b].oI,
                               (long long)lay[b].oT, (long long)lay[b].oW, lay[b].item0, lay[b].tile0});
        for (const auto& cl : bt.classes) sig.insert(sig.end(), {cl[0], cl[1], cl[2]});
    }
    // a run with batches of both precisions launches its FP64 batch on the
    // side stream, beside the FP32 one (the two touch disjoint partials;
    // k_lag_sum joins them); not while profiling, whose events time the
    // launches one after another on the main stream
    bool has32 = false, has64 = false;
    for (const LagBatch& bt : bts) (bt.dbl ? has64 : has32) = true;
    const bool fork = has32 && has64 && !c->prof;
    if (fork) {
        if (!c->side) KCU(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        if (!c->fork_ev) KCU(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
        if (!c->join_ev) KCU(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
    }
    // the upload from pinned staging, the launches and the copy back replay
    // as one graph (the copy reads the staging buffer when the graph runs)
    auto issue = [&]() -> int {
        KCU(cudaMemcpyAsync(dbase, h, bytes, cudaMemcpyHostToDevice, c->stream));
        // the staging buffer is free again once this copy is done (inside a
        // graph: an event node that records when the replayed copy is done),
        // so the host can stage the next chunk while these launches run
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        KCU(cudaStreamIsCapturing(c->stream, &cs));
        KCU(cudaEventRecordWithFlags(c->staging_ev, c->stream,
                                     cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                         : cudaEventRecordDefault));
        if (fork) {
            KCU(cudaEventRecord(c->fork_ev, c->stream));
            KCU(cudaStreamWaitEvent(c->side, c->fork_ev, 0));
        }
        for (size_t b = 0; b < bts.size(); ++b) {
            const LagBatch& bt = bts[b];
            const size_t nt = std::max<size_t>(bt.tiles.size(), 1);
            const cudaStream_t ls = (fork && bt.dbl) ? c->side : c->stream;
            for (const auto& cl : bt.classes) {
                cudaEvent_t ev = prof_start(c);
                if (bt.dbl) {
                    // fewer tiles than SMs: a warp slice per CTA, so that the
                    // FP64 points spread over kLagSlices times as many SMs
                    const bool sl = cl[2] < c->nsm;
                    const LagJob<double> j{(const LagItem<double>*)(dbase + lay[b].oI), (const LagTile*)(dbase + lay[b].oT),
                                           cl[1], cl[2], sl ? cl[2] * kLagSlices : std::min(cl[2], c->nsm * 8),
                                           sl ? 32 : 256, (const double*)(dbase + lay[b].oW),
                                           part + 2 * (size_t)lay[b].tile0};
                    KCU(launch_lag<double>(bt.d, cl[0], j, ls));
                } else {
                    const LagJob<float> j{(const LagItem<float>*)(dbase + lay[b].oI), (const LagTile*)(dbase + lay[b].oT),
                                          cl[1], cl[2], std::min(cl[2], c->nsm * 8), 256,
                                          (const float*)(dbase + lay[b].oW), part + 2 * (size_t)lay[b].tile0};
                    KCU(launch_lag<float>(bt.d, cl[0], j, ls));
                }
                prof_stop(c, ev, bt.dbl ? "lag_f64" : "lag_f32", bt.by * cl[2] / nt, bt.fl * cl[2] / nt);
            }
        }
        if (fork) {
            KCU(cudaEventRecord(c->join_ev, c->side));
            KCU(cudaStreamWaitEvent(c->stream, c->join_ev, 0));
        }
        cudaEvent_t es = prof_start(c);
        KCU(launch_lag_sum((const LagSum*)(dbase + oS), nit, part, dout, c->stream));
        prof_stop(c, es, "lag_sum", 16.0 * ntl, 2.0 * ntl);
        KCU(cudaMemcpyAsync((double*)c->h_out.p + off, dout, sizeof(double) * need, cudaMemcpyDeviceToHost, c->stream));
        return KDEFFT_OK;
    };
    KCHK(run_graph(c, sig, issue));
    c->staging_free = false;
    c->h2d += (int64_t)bytes;
    c->d2h += (int64_t)(sizeof(double) * need);
    for (size_t b = 0; b < bts.size(); ++b) {
        kdefft_ctx_s::PendingRead pr{&rs, std::move(bts[b].pairs), off + 2 * (size_t)lay[b].item0};
        c->pend_reads.push_back(std::move(pr));
    }
    c->hout_used += need;
    bts.clear();
    prof_flush(c);
    return KDEFFT_OK;
}

// One batch of work items through the chosen engine: the fused cluster
// kernel (d = 2) when allowed and the work fits, else the multi-pass path
// with tile capacity kb.cap; radix plans capped at kb.maxr.
template <typename real>
static int run_knobs(kdefft_ctx c, std::vector<Item<real>>& items, int d, const kdefft_ctx_s::Knobs& kb,
                     std::vector<double>& out) {
    for (Item<real>& it : items) {
        int P[MAXD] = {0};
        for (int k = 0; k < d; ++k) P[k] = it.ax[k].P;
        KCHK(fill_axes(c, d, P, it, kb.maxr));
    }
    int fr = KDEFFT_ERR_UNSUPPORTED;
    if (d == 2 && kb.fused) fr = launch_fused<real>(c, items, out.data());
    if (fr == KDEFFT_ERR_UNSUPPORTED) {
        PassLists pl;
        for (size_t i = 0; i < items.size(); ++i) tile_item(items[i], (int)i, kb.cap, pl);
        KCHK(launch_items<real>(c, items, pl, d, out.data()));
    } else if (fr != KDEFFT_OK) {
        return fr;
    }
    return KDEFFT_OK;
}

// Autotuner: the first batch of a shape (dimension, precision, number of
// items, largest padded size, largest support; the last three rounded up to
// powers of two) runs once per candidate -- engine (fused / multi-pass),
// multi-pass tile capacity (1/2, 1, 3/2 of the default), radix cap (32 / 16
// in FP32, 16 / 8 in FP64) -- timed on the host clock around the whole batch
// (staging, launches, copies, wait); the fastest is cached for the shape and
// its results are the batch's.  Off: the default knobs.
template <typename real>
static int dispatch_batch(kdefft_ctx c, std::vector<Item<real>>& items, int d, int cap, std::vector<double>& out) {
    const bool dbl = sizeof(real) == 8;
    kdefft_ctx_s::Knobs def{(d == 2 && c->fused) ? 1 : 0, cap, dbl ? 16 : 32};
    if (!c->autotune) return run_knobs<real>(c, items, d, def, out);
    auto pow2 = [](long long v) {
        long long p = 1;
        while (p < v) p *= 2;
        return p;
    };
    long long pmax = 0, smax = 0;
    for (const Item<real>& it : items) {
        long long sp = 1;
        for (int k = 0; k < d; ++k) {
            pmax = std::max<long long>(pmax, it.ax[k].P);
            sp *= it.S[k];
        }
        smax = std::max(smax, sp);
    }
    const std::array<long long, 5> key{d, dbl ? 1 : 0, pow2((long long)items.size()), pow2(pmax), pow2(smax)};
    auto hit = c->tuned.find(key);
    if (hit != c->tuned.end()) return run_knobs<real>(c, items, d, hit->second, out);
    std::vector<kdefft_ctx_s::Knobs> cand;
    const int radix[2] = {dbl ? 16 : 32, dbl ? 8 : 16};
    if (d == 2 && c->fused)
        for (int r : radix) cand.push_back({1, cap, r});
    for (int cm : {2, 4, 6})   // tile capacity cap / 2, cap, 3 cap / 2
        for (int r : radix) {
            const int cc = cap * cm / 4;
            // every line fits a batch, and the largest pass's shared memory
            // (two padded ping-pong buffers, twiddles, staged spectrum) fits a CTA
            const size_t sm = (2 * sizeof(real)) * (size_t)(2 * (cc + cc / 16 + 1) + pmax) + sizeof(real) * cc;
            if (cc < pmax || sm > 220 * 1024) continue;
            cand.push_back({0, cc, r});
        }
    double best_t = INFINITY;
    kdefft_ctx_s::Knobs best = def;
    std::vector<double> o(out.size());
    for (const auto& kb : cand) {
        // one untimed run (first-use set-up), one timed
        const int r0 = run_knobs<real>(c, items, d, kb, o);
        if (r0 == KDEFFT_ERR_UNSUPPORTED) continue;
        KCHK(r0);
        const auto t0 = std::chrono::steady_clock::now();
        KCHK(run_knobs<real>(c, items, d, kb, o));
        const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (t < best_t) {
            best_t = t;
            best = kb;
            out = o;
        }
    }
    if (!std::isfinite(best_t)) return run_knobs<real>(c, items, d, def, out);
    c->tuned[key] = best;
    c->keys_tuned++;
    return KDEFFT_OK;
}

// The selected grids of one precision: lag-domain pairs are built into lagq
// (issued by the caller with the other precision's), the rest run the FFT
// route here.
template <typename real>
static int run_requests(kdefft_ctx c, ReqSet& rs, const std::vector<int>& sel, std::vector<LagBatch>& lagq) {
    if (sel.empty()) return KDEFFT_OK;
    const int d = rs.grids[sel[0]].ds->d;
    HermiteIndex& hx = hindex();
    // pair consecutive selected grids that share dataset, covariances and plan
    std::vector<std::pair<int, int>> pairs;
    for (size_t u = 0; u < sel.size();) {
        const GridReq& a = rs.grids[sel[u]];
        if (u + 1 < sel.size()) {
            const GridReq& b = rs.grids[sel[u + 1]];
            if (b.ds == a.ds && b.spec == a.spec && std::memcmp(a.L, b.L, sizeof(a.L)) == 0 &&
                std::memcmp(a.P, b.P, sizeof(a.P)) == 0) {
                pairs.push_back({sel[u], sel[u + 1]});
                u += 2;
                continue;
            }
        }
        pairs.push_back({sel[u], -1});
        u += 1;
    }
    const int cap = cap_elems(sizeof(real) == 8);
    // lag-domain engine for the pairs it covers; the FFT route for the rest
    {
        std::vector<std::pair<int, int>> lagp, fftp;
        for (const auto& pr : pairs) (lag_eligible<real>(c, rs, pr) ? lagp : fftp).push_back(pr);
        if (!lagp.empty()) {
            const int lr = run_lag<real>(c, rs, lagp, lagq);
            if (lr == KDEFFT_ERR_UNSUPPORTED)
                fftp.insert(fftp.end(), lagp.begin(), lagp.end());   // autocorrelation box beyond MAXP
            else
                KCHK(lr);
        }
        pairs.swap(fftp);
        if (pairs.empty()) return KDEFFT_OK;
    }
    // count spectra first, all missing ones in one launch sequence
    {
        HostTimer hs(c, "host:spectra");
        std::vector<std::pair<kdefft_ds, std::array<int, 4>>> need;
        std::set<std::pair<kdefft_ds, std::array<int, 4>>> seen;
        for (const auto& pr : pairs) {
            const GridReq& g = rs.grids[pr.first];
            std::array<int, 4> P{g.P[0], g.P[1], g.P[2], g.P[3]};
            if (seen.insert({g.ds, P}).second) need.push_back({g.ds, P});
        }
        KCHK(ensure_spectra<real>(c, need));
    }
    // scratch budget per launch: split the items into batches
    const long long budget = 1LL << 28;   // complex elements (2 GiB at FP32)
    size_t pi = 0;
    while (pi < pairs.size()) {
        std::vector<Item<real>> items;
        std::vector<std::pair<int, int>> batch;
        long long scratch = 0;
        {
            HostTimer hb(c, "host:build");
            while (pi < pairs.size()) {
                const auto pr = pairs[pi];
                const GridReq& g = rs.grids[pr.first];
                const KSpec& sp = rs.specs[g.spec];
                Item<real> it;
                std::memset(&it, 0, sizeof(it));
                it.d = d;
                it.kind = 0;
                KCHK(fill_axes(c, d, g.P, it));
                long long ptot = 1;
                for (int k = 0; k < d; ++k) {
                    it.S[k] = 2 * g.L[k] + 1;
                    it.off[k] = g.L[k];
                    it.delta[k] = g.ds->delta[k];
                    ptot *= g.P[k];
                }
                it.nsig = sp.nsig;
                for (int s = 0; s < sp.nsig; ++s) {
                    Mat inv;
                    double det;
                    if (!spd_inv_det(sp.sig[s], inv, det))
                        return fail(KDEFFT_ERR_NOT_SPD, "a kernel covariance is not positive definite");
                    for (int a = 0; a < d; ++a)
                        for (int b = 0; b < d; ++b) it.lam[s][a * MAXD + b] = inv(a, b);
                    it.nrm[s] = std::pow(2.0 * M_PI, -0.5 * d) / std::sqrt(det);
                }
                int R = 0;
                const int gi[2] = {pr.first, pr.second};
                for (int h = 0; h < 2; ++h) {
                    if (gi[h] < 0) {
                        it.nterm[h] = 0;
                        continue;
                    }
                    const TermVec& tl = rs.grids[gi[h]].terms;
                    if ((int)tl.size() > MAXTERM) return fail(KDEFFT_ERR_UNSUPPORTED, "too many kernel terms");
                    it.nterm[h] = tl.size();
                    for (int m = 0; m < tl.size(); ++m) {
                        int o = 0;
                        for (int k = 0; k < d; ++k) o += tl[m].alpha[k];
                        if (o > kRmax[d]) return fail(KDEFFT_ERR_UNSUPPORTED, "derivative order too high for d");
                        R = std::max(R, o);
                        const int hidx = hx.idx(d, tl[m].alpha);
                        it.tsig[h][m] = (short)tl[m].sig;
                        it.the[h][m] = (short)hidx;
                        it.tw8[h][m] = (real)(((o & 1) ? -1.0 : 1.0) * tl[m].w);
                    }
                }
                it.R = R;
                auto sp_it = g.ds->spectra.find(spectrum_key(g.ds, g.P, sizeof(real)));
                if (sp_it == g.ds->spectra.end()) return fail(KDEFFT_ERR_CUDA, "count spectrum missing");
                it.spec = (const real*)sp_it->second->p;
                const double nn = (double)g.ds->n;
                it.scale = 1.0 / (nn * nn * (double)ptot);
                // would this item overflow the multi-pass scratch budget?
                const long long need = scratch_need(it);
                if (!items.empty() && scratch + need > budget) break;
                scratch += need;
                items.push_back(it);
                batch.push_back(pr);
                ++pi;
            }
        }
        std::vector<double> out(2 * items.size());
        KCHK(dispatch_batch<real>(c, items, d, cap, out));
        for (size_t i = 0; i < batch.size(); ++i) {
            rs.grids[batch[i].first].value = out[2 * i];
            if (batch[i].second >= 0) rs.grids[batch[i].second].value = out[2 * i + 1];
        }
    }
    return KDEFFT_OK;
}

// Evaluate all grids: FP64 datasets and grids marked fp64 in double, the
// rest in float.
static int run(kdefft_ctx c, ReqSet& rs) {
    if (rs.grids.empty()) return KDEFFT_OK;
    HostTimer ht(c, "host:run");
    std::vector<int> s32, s64;
    for (size_t i = 0; i < rs.grids.size(); ++i) {
        const GridReq& g = rs.grids[i];
        ((g.fp64 || g.ds->opts.precision == KDEFFT_FP64) ? s64 : s32).push_back((int)i);
    }
    std::vector<LagBatch> lagq;
    int r = run_requests<double>(c, rs, s64, lagq);
    if (r == KDEFFT_OK) r = run_requests<float>(c, rs, s32, lagq);
    // the lag batches of both precisions: one upload, one launch sequence,
    // one copy back, one wait (also on an error, as the pending reads point
    // into rs)
    if (r == KDEFFT_OK) r = issue_lag(c, rs, lagq);
    const int f = flush_reads(c);
    return r != KDEFFT_OK ? r : f;
}

// ============================================================ objective assembly
static void assemble_lscv(kdefft_ds ds, const Mat& H, const GridReq* g, double* val, double* grad) {
    const int d = ds->d;
    const double n = (double)ds->n;
    Mat inv;
    double det;
    spd_inv_det(H, inv, det);
    const double k0 = std::pow(2.0 * M_PI, -0.5 * d) / std::sqrt(det);
    int gi = 0;
    double c0;
    if (!ds->opts.exact_loo) {
        *val = g[0].value + 2.0 * k0 / n;
        gi = 1;
        c0 = 2.0 / n;
    } else {
        *val = g[0].value - 2.0 * n / (n - 1.0) * g[1].value + 2.0 / (n - 1.0) * k0;
        gi = 2;
        c0 = 2.0 / (n - 1.0);
    }
    if (grad) {
        for (int a = 0; a < d; ++a)
            for (int b = a; b < d; ++b) {
                const double tie = (a == b) ? 1.0 : 2.0;
                const double v = g[gi++].value + c0 * tie * (-0.5 * k0 * inv(a, b));
                grad[a * d + b] = grad[b * d + a] = v;
            }
    }
}

static void assemble_scv(kdefft_ds ds, const Mat& H, const GridReq* g, bool split64, double c2g, double* val,
                         double* grad) {
    const int d = ds->d;
    const double n = (double)ds->n;
    Mat inv;
    double det;
    spd_inv_det(H, inv, det);
    const double r0 = std::pow(4.0 * M_PI, -0.5 * d) / std::sqrt(det);
    *val = r0 / n + (split64 ? (g[0].value - 2.0 * g[1].value + c2g) : g[0].value);
    if (grad) {
        int gi = split64 ? 2 : 1;
        for (int a = 0; a < d; ++a)
            for (int b = a; b < d; ++b) {
                const double tie = (a == b) ? 1.0 : 2.0;
                const double v = g[gi++].value + tie * (-0.5 * r0 * inv(a, b)) / n;
                grad[a * d + b] = grad[b * d + a] = v;
            }
    }
}

// psi_4 unique values -> Kronecker vector (Sec. 5 ordering)
// Position in the Kronecker-ordered d^r vector -> index of its multi-index
// in `alphas` (a flat index i_1 + d i_2 + ... counts how often each axis
// occurs); one map serves every bandwidth of a call.
static std::vector<int> kron_map(int d, int r, const std::vector<MultiIndex>& alphas) {
    std::vector<int> code(9 * 9 * 9 * 9, -1);
    for (size_t i = 0; i < alphas.size(); ++i) code[HermiteIndex::key(d, alphas[i].a)] = (int)i;
    long long total = 1;
    for (int i = 0; i < r; ++i) total *= d;
    std::vector<int> map((size_t)total);
    for (long long pos = 0; pos < total; ++pos) {
        int al[MAXD] = {0, 0, 0, 0};
        long long p = pos;
        for (int i = 0; i < r; ++i) {
            al[p % d]++;
            p /= d;
        }
        map[(size_t)pos] = code[HermiteIndex::key(d, al)];
    }
    return map;
}

static void kron_expand(const std::vector<int>& map, const GridReq* g, double* out) {
    for (size_t pos = 0; pos < map.size(); ++pos) out[pos] = g[map[pos]].value;
}

static void assemble_pi(kdefft_ds ds, const Mat& H, const double* psi4, double* val, double* grad) {
    const int d = ds->d;
    const double n = (double)ds->n;
    Mat inv;
    double det;
    spd_inv_det(H, inv, det);
    const double r0 = std::pow(4.0 * M_PI, -0.5 * d) / std::sqrt(det);
    auto T = [&](int a, int b, int c, int e) { return psi4[((a * d + b) * d + c) * d + e]; };
    double quad = 0.0;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b)
            for (int c = 0; c < d; ++c)
                for (int e = 0; e < d; ++e) quad += H(a, b) * H(c, e) * T(a, b, c, e);
    *val = r0 / n + 0.25 * quad;
    if (grad) {
        for (int a = 0; a < d; ++a)
            for (int b = a; b < d; ++b) {
                double half = 0.0;
                for (int c = 0; c < d; ++c)
                    for (int e = 0; e < d; ++e) half += H(c, e) * T(a, b, c, e);
                half *= 0.5;
                const double tie = (a == b) ? 1.0 : 2.0;
                const double v = tie * (half - 0.5 * r0 * inv(a, b) / n);
                grad[a * d + b] = grad[b * d + a] = v;
            }
    }
}

static int write_out(kdefft_ctx c, double* dst, const double* src, size_t count) {
    if (!dst || count == 0) return KDEFFT_OK;
    if (is_device_ptr(dst)) {
        c->h2d += (int64_t)(sizeof(double) * count);
        KCU(cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
        KCU(cudaStreamSynchronize(c->stream));
    } else {
        std::memcpy(dst, src, sizeof(double) * count);
    }
    return KDEFFT_OK;
}

// ============================================================ C ABI
// Handles the library has handed out and not yet destroyed: a destroy call
// checks its handle here before touching it, so that a second destroy of the
// same handle is an error, not a use after free.
static std::mutex g_live_mu;
static std::set<const void*> g_live;
static void live_add(const void* h) {
    std::lock_guard<std::mutex> g(g_live_mu);
    g_live.insert(h);
}
static bool live_take(const void* h) {
    std::lock_guard<std::mutex> g(g_live_mu);
    return g_live.erase(h) > 0;
}

// The dataset's blocks go back to the context's cache, whose reuse is ordered
// by the context's stream, so work still queued on them needs no wait here.
static void ds_free(kdefft_ds ds) {
    HostTimer ht(ds->ctx, "host:close");
    cudaSetDevice(ds->ctx->device);
    ds->counts.release();
    ds->counts_i.release();
    ds->counts64.release();
    ds->ac64.release();
    ds->ac32.release();
    for (auto& kv : ds->spectra) kv.second->release();
    delete ds;
}

extern "C" {

int kdefft_opts_default(kdefft_opts* o) {
    if (!o) return fail(KDEFFT_ERR_ARG, "opts is NULL");
    std::memset(o, 0, sizeof(*o));
    o->tau = 3.7;
    o->L_basis = KDEFFT_L_AUTO;
    o->P_rule = KDEFFT_P_MINIMAL;
    o->exact_loo = 0;
    o->precision = KDEFFT_FP32;
    o->binning = KDEFFT_BIN_LINEAR;
    o->outside_policy = KDEFFT_OUTSIDE_ERROR;
    return KDEFFT_OK;
}

const char* kdefft_strerror(int code) {
    switch (code) {
        case KDEFFT_OK: return "ok";
        case KDEFFT_ERR_ARG: return "invalid argument";
        case KDEFFT_ERR_NOT_SPD: return "matrix not symmetric positive definite";
        case KDEFFT_ERR_OUTSIDE_GRID: return "sample point outside the grid";
        case KDEFFT_ERR_CUDA: return "CUDA error";
        case KDEFFT_ERR_ALLOC: return "allocation failed";
        case KDEFFT_ERR_TIMEOUT: return "device wait timed out";
        case KDEFFT_ERR_UNSUPPORTED: return "unsupported size";
        default: return "unknown error";
    }
}

const char* kdefft_last_error(void) { return g_err.c_str(); }

int kdefft_create(kdefft_ctx* out, int device, void* stream) {
    if (!out) return fail(KDEFFT_ERR_ARG, "ctx is NULL");
    *out = nullptr;
    int ndev = 0;
    KCU(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(KDEFFT_ERR_ARG, "no such CUDA device");
    KCU(cudaSetDevice(device));
    auto c = new kdefft_ctx_s();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return fail(KDEFFT_ERR_CUDA, "cudaGetDeviceProperties failed");
    }
    c->nsm = prop.multiProcessorCount;
    for (DevBuf* b : {&c->tw32, &c->tw64, &c->twdf, &c->scratch, &c->partial, &c->items, &c->tiles, &c->out,
                      &c->sel_buf, &c->binfix, &c->acbuf[0], &c->acbuf[1], &c->acjobs, &c->binjobs, &c->kdebuf,
                      &c->specjobs})
        b->gen = &c->buf_gen;
    c->h_items.gen = &c->buf_gen;
    c->h_out.gen = &c->buf_gen;
    c->h_binres.gen = &c->buf_gen;
    if (cudaEventCreateWithFlags(&c->staging_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->acjobs_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->specjobs_ev, cudaEventDisableTiming) != cudaSuccess) {
        delete c;
        return fail(KDEFFT_ERR_CUDA, "event creation failed");
    }
    if (cudaMalloc(&c->errflag, sizeof(int)) != cudaSuccess || cudaMemset(c->errflag, 0, sizeof(int)) != cudaSuccess) {
        delete c;
        return fail(KDEFFT_ERR_ALLOC, "error flag allocation failed");
    }
    int r = upload_tables();
    if (r == KDEFFT_OK && prepare_binning() != cudaSuccess) r = fail(KDEFFT_ERR_CUDA, "binning kernel attributes");
    if (r == KDEFFT_OK && prepare_kernels() != cudaSuccess) r = fail(KDEFFT_ERR_CUDA, "kernel shared-memory attributes");
    if (r != KDEFFT_OK) {
        delete c;
        return r;
    }
    *out = c;
    live_add(c);
    return KDEFFT_OK;
}

int kdefft_set_engine(kdefft_ctx c, int engine) {
    if (!c) return fail(KDEFFT_ERR_ARG, "NULL context");
    if (engine != KDEFFT_ENGINE_AUTO && engine != KDEFFT_ENGINE_MULTIPASS && engine != KDEFFT_ENGINE_HOST_SELECT &&
        engine != KDEFFT_ENGINE_FFT)
        return fail(KDEFFT_ERR_ARG, "unknown engine");
    c->fused = (engine != KDEFFT_ENGINE_MULTIPASS);
    c->device_select = (engine == KDEFFT_ENGINE_AUTO || engine == KDEFFT_ENGINE_FFT);
    c->lag = (engine == KDEFFT_ENGINE_AUTO || engine == KDEFFT_ENGINE_HOST_SELECT);
    return KDEFFT_OK;
}

int kdefft_autocorr(kdefft_ds ds, const int* A, double* out) {
    if (!ds || !A || !out) return fail(KDEFFT_ERR_ARG, "NULL argument");
    kdefft_ctx c = ds->ctx;
    const int d = ds->d;
    for (int k = 0; k < d; ++k)
        if (A[k] < 0 || A[k] > ds->M[k] - 1) return fail(KDEFFT_ERR_ARG, "A_k must be in [0, M_k - 1]");
    KCU(cudaSetDevice(c->device));
    std::array<int, 4> need{0, 0, 0, 0};
    for (int k = 0; k < d; ++k) need[k] = A[k];
    const int r = ensure_autocorr_many(c, {{ds, need}});
    if (r == KDEFFT_ERR_UNSUPPORTED) return fail(r, "the padding for this box exceeds 4096");
    KCHK(r);
    long long nbox = 1;
    for (int k = 0; k < d; ++k) nbox *= (k == 0) ? (ds->acA[0] + 1) : (2 * ds->acA[k] + 1);
    std::vector<double> full((size_t)nbox);
    KCU(cudaMemcpyAsync(full.data(), ds->ac64.p, sizeof(double) * nbox, cudaMemcpyDeviceToHost, c->stream));
    KCU(cudaStreamSynchronize(c->stream));
    c->d2h += (int64_t)(sizeof(double) * nbox);
    // the requested sub-box, same layout
    long long nout = 1;
    for (int k = 0; k < d; ++k) nout *= (k == 0) ? (A[0] + 1) : (2 * A[k] + 1);
    for (long long f = 0; f < nout; ++f) {
        long long g = f, src = 0;
        int j[4] = {0, 0, 0, 0};
        j[0] = (int)(g % (A[0] + 1));
        g /= (A[0] + 1);
        for (int k = 1; k < d; ++k) {
            j[k] = (int)(g % (2 * A[k] + 1)) - A[k];
            g /= (2 * A[k] + 1);
        }
        for (int k = d - 1; k >= 1; --k) src = src * (2 * ds->acA[k] + 1) + (j[k] + ds->acA[k]);
        src = src * (ds->acA[0] + 1) + j[0];
        out[f] = full[(size_t)src];
    }
    return KDEFFT_OK;
}

int kdefft_set_autotune(kdefft_ctx c, int on) {
    if (!c) return fail(KDEFFT_ERR_ARG, "NULL context");
    c->autotune = (on != 0);
    return KDEFFT_OK;
}

int kdefft_set_graphs(kdefft_ctx c, int on) {
    if (!c) return fail(KDEFFT_ERR_ARG, "NULL context");
    c->graphs = (on != 0);
    return KDEFFT_OK;
}

int kdefft_set_search_record(kdefft_ctx c, double* rec, int64_t rec_len, int cap) {
    if (!c) return fail(KDEFFT_ERR_ARG, "NULL context");
    if (!rec) {
        c->rec = nullptr;
        c->rec_len = 0;
        c->rec_cap = 0;
        return KDEFFT_OK;
    }
    if (cap < 1 || rec_len < (int64_t)cap * SEL_REC) return fail(KDEFFT_ERR_ARG, "record buffer too small for one start");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, rec) != cudaSuccess) {
        cudaGetLastError();
        return fail(KDEFFT_ERR_ARG, "record buffer is not device memory");
    }
    if (a.type != cudaMemoryTypeDevice || a.device != c->device)
        return fail(KDEFFT_ERR_ARG, "record buffer is not device memory of the context's GPU");
    c->rec = rec;
    c->rec_len = rec_len;
    c->rec_cap = cap;
    return KDEFFT_OK;
}

int kdefft_runtime_stats(kdefft_ctx c, int64_t* shapes_tuned, int64_t* graphs_captured, int64_t* graph_replays) {
    if (!c) return fail(KDEFFT_ERR_ARG, "NULL context");
    if (shapes_tuned) *shapes_tuned = c->keys_tuned;
    if (graphs_captured) *graphs_captured = c->graphs_captured;
    if (graph_replays) *graph_replays = c->graph_replays;
    return KDEFFT_OK;
}

int kdefft_memory_stats(kdefft_ctx c, int64_t* cached_bytes, int64_t* hits, int64_t* misses) {
    if (!c) return fail(KDEFFT_ERR_ARG, "NULL context");
    if (cached_bytes) *cached_bytes = (int64_t)c->cache.bytes;
    if (hits) *hits = c->cache.hits;
    if (misses) *misses = c->cache.misses;
    return KDEFFT_OK;
}

int kdefft_trim(kdefft_ctx c) {
    if (!c) return fail(KDEFFT_ERR_ARG, "NULL context");
    KCU(cudaSetDevice(c->device));
    KCU(cudaStreamSynchronize(c->stream));
    c->cache.trim();
    return KDEFFT_OK;
}

int kdefft_profile(kdefft_ctx c, int mode) {
    if (!c) return fail(KDEFFT_ERR_ARG, "NULL context");
    if (mode == 1 || mode == 0) {
        c->kstat.clear();
        c->launches = c->h2d = c->d2h = 0;
    }
    c->prof = (mode != 0);
    return KDEFFT_OK;
}

int kdefft_profile_read(kdefft_ctx c, kdefft_kstat* out, int cap, int* count, int64_t* launches, int64_t* h2d_bytes,
                        int64_t* d2h_bytes) {
    if (!c) return fail(KDEFFT_ERR_ARG, "NULL context");
    int i = 0;
    for (auto& kv : c->kstat) {
        if (out && i < cap) {
            std::memset(&out[i], 0, sizeof(out[i]));
            std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = kv.second.launches;
            out[i].ms = kv.second.ms;
            out[i].bytes = kv.second.bytes;
            out[i].flops = kv.second.flops;
        }
        ++i;
    }
    if (count) *count = i;
    if (launches) *launches = c->launches;
    if (h2d_bytes) *h2d_bytes = c->h2d;
    if (d2h_bytes) *d2h_bytes = c->d2h;
    return KDEFFT_OK;
}

int kdefft_destroy(kdefft_ctx c) {
    if (!c) return KDEFFT_OK;
    if (!live_take(c)) return fail(KDEFFT_ERR_ARG, "unknown or already destroyed context");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (kdefft_ds ds : c->datasets) {
        live_take(ds);
        ds_free(ds);
    }
    c->datasets.clear();
    c->cache.trim();
    c->tw32.release();
    c->tw64.release();
    c->scratch.release();
    c->partial.release();
    c->items.release();
    c->tiles.release();
    c->out.release();
    c->sel_buf.release();
    c->binfix.release();
    c->acbuf[0].release();
    c->acbuf[1].release();
    c->acjobs.release();
    c->binjobs.release();
    c->kdebuf.release();
    c->h_items.release();
    c->h_out.release();
    for (auto& p : c->pending) {
        c->evpool.push_back(p.a);
        c->evpool.push_back(p.b);
    }
    for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
    for (auto& kv : c->gcache) cudaGraphExecDestroy(kv.second.exec);
    c->gcache.clear();
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->staging_ev) cudaEventDestroy(c->staging_ev);
    if (c->acjobs_ev) cudaEventDestroy(c->acjobs_ev);
    if (c->specjobs_ev) cudaEventDestroy(c->specjobs_ev);
    c->h_acjobs.release();
    c->h_specjobs.release();
    c->h_sel.release();
    c->h_binres.release();
    if (c->errflag) cudaFree(c->errflag);
    delete c;
    return KDEFFT_OK;
}

// Eq. 8's leave-one-out sum over j != i carries 1/(n (n - 1)): it has no
// value for a single point
static const char* const kLooNeedsTwo = "exact leave-one-out (Eq. 8) needs n >= 2";

int kdefft_bin(kdefft_ctx c, const double* X, int64_t n, int d, const double* lo, const double* hi,
               const int64_t* M, const kdefft_opts* opts, kdefft_ds* out) {
    if (!c || !out || !lo || !hi || !M) return fail(KDEFFT_ERR_ARG, "NULL argument");
    HostTimer ht(c, "host:bin");
    *out = nullptr;
    if (d < 1 || d > 4) return fail(KDEFFT_ERR_ARG, "d must be 1..4");
    if (n < 1 || (!X)) return fail(KDEFFT_ERR_ARG, "need n >= 1 samples");
    kdefft_opts o;
    if (opts)
        o = *opts;
    else
        kdefft_opts_default(&o);
    if (!(o.tau > 0.0)) return fail(KDEFFT_ERR_ARG, "tau must be positive");
    if (o.exact_loo && n < 2) return fail(KDEFFT_ERR_ARG, kLooNeedsTwo);
    KCU(cudaSetDevice(c->device));
    std::unique_ptr<kdefft_ds_s> ds(new kdefft_ds_s());
    ds->ctx = c;
    attach_cache(*ds, c);
    ds->d = d;
    ds->n = n;
    ds->opts = o;
    GridDesc g;
    std::memset(&g, 0, sizeof(g));
    g.d = d;
    ds->ncells = 1;
    for (int k = 0; k < d; ++k) {
        if (M[k] < 2 || M[k] > (1 << 20)) return fail(KDEFFT_ERR_ARG, "M_k must be in [2, 2^20]");
        if (!(hi[k] > lo[k]) || !std::isfinite(lo[k]) || !std::isfinite(hi[k]))
            return fail(KDEFFT_ERR_ARG, "need lo_k < hi_k, finite");
        ds->lo[k] = lo[k];
        ds->hi[k] = hi[k];
        ds->M[k] = M[k];
        ds->delta[k] = (hi[k] - lo[k]) / (double)(M[k] - 1);   // Eq. 16
        g.lo[k] = ds->lo[k];
        g.hi[k] = ds->hi[k];
        g.delta[k] = ds->delta[k];
        g.M[k] = M[k];
        ds->ncells *= M[k];
    }
    if (ds->ncells > (1LL << 31)) return fail(KDEFFT_ERR_UNSUPPORTED, "grid too large");
    // sample on the device
    DevBuf xbuf(&c->cache);
    const double* dX = X;
    if (!is_device_ptr(X)) {
        KCHK(xbuf.ensure(sizeof(double) * n * d));
        KCU(cudaMemcpyAsync(xbuf.p, X, sizeof(double) * n * d, cudaMemcpyHostToDevice, c->stream));
        c->h2d += (int64_t)(sizeof(double) * n * d);
        dX = (const double*)xbuf.p;
    }
    // outside counter | block partials of the moments
    const int mblk = moments_blocks(n, c->nsm);
    const int nv = d + d * d;
    DevBuf misc(&c->cache);
    KCHK(misc.ensure(sizeof(double) * (16 + (size_t)mblk * nv)));
    unsigned long long* dOut = (unsigned long long*)misc.p;
    double* dPart = (double*)misc.p + 16;
    const bool dbl = o.precision == KDEFFT_FP64;
    // covariance for the normal-scale start point, in one pass shifted by the
    // grid's centre (block partials summed in block order: the same start
    // point from run to run)
    Shift sh{};
    for (int k = 0; k < d; ++k) sh.s[k] = 0.5 * (lo[k] + hi[k]);
    unsigned long long nout = 0;
    std::vector<double> part((size_t)mblk * nv);
    if (!dbl && o.binning != KDEFFT_BIN_SIMPLE) {
        // FP32 linear binning: the launch sequence (zeroing, binning, fixed
        // point to FP32, moments, copies of the outside count and the moment
        // partials to pinned memory) replays as a CUDA graph when its
        // pointers and sizes repeat
        int K = 32;   // fixed point with K fractional bits; a cell's total (<= n 2^K) stays below 2^63
        while (K > 8 && (double)n * std::ldexp(1.0, K) >= std::ldexp(1.0, 63)) --K;
        DevBuf& fix = c->binfix;
        KCHK(fix.ensure(8 * (size_t)ds->ncells));
        KCHK(ds->counts.ensure(4 * (size_t)ds->ncells));
        // the outside counter and the moment partials come back in one copy
        // of the whole work buffer (counter at 0, partials from 16)
        const size_t nres = 16 + (size_t)mblk * nv;
        KCHK(c->h_binres.ensure(sizeof(double) * nres));
        double* hres = (double*)c->h_binres.p;
        std::vector<long long> sig = {4, (long long)(uintptr_t)dX, n, d, K, (long long)(uintptr_t)fix.p,
                                      (long long)(uintptr_t)ds->counts.p, (long long)(uintptr_t)misc.p,
                                      (long long)(uintptr_t)hres, mblk, ds->ncells, c->nsm};
        for (int k = 0; k < d; ++k) {
            long long bits[3];
            std::memcpy(&bits[0], &g.lo[k], 8);
            std::memcpy(&bits[1], &g.hi[k], 8);
            std::memcpy(&bits[2], &g.delta[k], 8);
            sig.insert(sig.end(), {bits[0], bits[1], bits[2], g.M[k]});
        }
        auto issue = [&]() -> int {
            KCU(cudaMemsetAsync(misc.p, 0, sizeof(double) * 16, c->stream));
            KCU(cudaMemsetAsync(fix.p, 0, 8 * (size_t)ds->ncells, c->stream));
            cudaEvent_t evb = prof_start(c);
            c->launches++;   // the fixed-point-to-FP32 conversion
            KCU(launch_bin_linear<unsigned long long>(dX, n, g, (unsigned long long*)fix.p, ds->ncells, dOut,
                                                      std::ldexp(1.0, K), c->nsm, c->stream));
            KCU(launch_fix_to_f32((const unsigned long long*)fix.p, (float*)ds->counts.p, ds->ncells,
                                  std::ldexp(1.0, -K), c->stream));
            prof_stop(c, evb, "bin", (double)n * d * 8.0 + (double)ds->ncells * 4.0, (double)n * (1 << d) * 2.0);
            c->launches += 1;
            KCU(launch_moments_shifted(dX, n, d, sh, dPart, c->nsm, c->stream));
            KCU(cudaMemcpyAsync(hres, misc.p, sizeof(double) * nres, cudaMemcpyDeviceToHost, c->stream));
            return KDEFFT_OK;
        };
        KCHK(run_graph(c, sig, issue));
        KCU(cudaStreamSynchronize(c->stream));
        std::memcpy(&nout, hres, sizeof(nout));
        std::memcpy(part.data(), hres + 16, sizeof(double) * mblk * nv);
    } else {
        KCU(cudaMemsetAsync(misc.p, 0, sizeof(double) * 16, c->stream));
        KCHK(ds->counts.ensure((dbl ? 8 : 4) * (size_t)ds->ncells));
        // only FP64 linear binning accumulates into the counts themselves; the
        // other paths write every cell from their own accumulators
        if (dbl && o.binning != KDEFFT_BIN_SIMPLE)
            KCU(cudaMemsetAsync(ds->counts.p, 0, 8 * (size_t)ds->ncells, c->stream));
        cudaEvent_t evb = prof_start(c);
        if (o.binning == KDEFFT_BIN_SIMPLE) {
            c->launches++;   // the integer-to-real conversion
            KCHK(ds->counts_i.ensure(4 * (size_t)ds->ncells));
            KCU(cudaMemsetAsync(ds->counts_i.p, 0, 4 * (size_t)ds->ncells, c->stream));
            KCU(launch_bin_simple(dX, n, g, (int*)ds->counts_i.p, ds->ncells, dOut, c->nsm, c->stream));
            if (dbl)
                KCU(launch_int_to_real<double>((int*)ds->counts_i.p, (double*)ds->counts.p, ds->ncells, c->stream));
            else
                KCU(launch_int_to_real<float>((int*)ds->counts_i.p, (float*)ds->counts.p, ds->ncells, c->stream));
        } else {
            KCU(launch_bin_linear<double>(dX, n, g, (double*)ds->counts.p, ds->ncells, dOut, 1.0, c->nsm, c->stream));
        }
        prof_stop(c, evb, "bin", (double)n * d * 8.0 + (double)ds->ncells * (dbl ? 8.0 : 4.0), (double)n * (1 << d) * 2.0);
        c->launches += 1;
        KCU(launch_moments_shifted(dX, n, d, sh, dPart, c->nsm, c->stream));
        KCU(cudaMemcpyAsync(&nout, dOut, sizeof(nout), cudaMemcpyDeviceToHost, c->stream));
        KCU(cudaMemcpyAsync(part.data(), dPart, sizeof(double) * mblk * nv, cudaMemcpyDeviceToHost, c->stream));
        KCU(cudaStreamSynchronize(c->stream));
    }
    double hs[20] = {0};
    for (int b = 0; b < mblk; ++b)
        for (int v = 0; v < nv; ++v) hs[v] += part[(size_t)b * nv + v];
    prof_flush(c);
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b)
            ds->cov[a * d + b] = (n > 1) ? (hs[d + a * d + b] - hs[a] * hs[b] / (double)n) / (double)(n - 1) : 0.0;
    if (nout > 0 && o.outside_policy == KDEFFT_OUTSIDE_ERROR)
        return fail(KDEFFT_ERR_OUTSIDE_GRID, std::to_string(nout) + " sample points outside the grid");
    ds->dropped = (int64_t)nout;
    xbuf.release();
    misc.release();
    *out = ds.release();
    c->datasets.push_back(*out);
    live_add(*out);
    return KDEFFT_OK;
}

int kdefft_bin_many(kdefft_ctx c, int nds, const double* const* X, const int64_t* n, int d, const double* lo,
                    const double* hi, const int64_t* M, const kdefft_opts* opts, kdefft_ds* out) {
    if (!c || !X || !n || !lo || !hi || !M || !out || nds < 1) return fail(KDEFFT_ERR_ARG, "NULL argument");
    HostTimer ht(c, "host:bin");
    if (d < 1 || d > 4) return fail(KDEFFT_ERR_ARG, "d must be 1..4");
    for (int i = 0; i < nds; ++i) out[i] = nullptr;
    kdefft_opts o;
    if (opts)
        o = *opts;
    else
        kdefft_opts_default(&o);
    if (!(o.tau > 0.0)) return fail(KDEFFT_ERR_ARG, "tau must be positive");
    if (o.precision != KDEFFT_FP32 || o.binning != KDEFFT_BIN_LINEAR) {
        // other precisions and rules: one dataset at a time
        for (int i = 0; i < nds; ++i) {
            const int r = kdefft_bin(c, X[i], n[i], d, lo + (size_t)i * d, hi + (size_t)i * d, M + (size_t)i * d, &o,
                                     &out[i]);
            if (r != KDEFFT_OK) {
                for (int j = 0; j < i; ++j) kdefft_ds_destroy(out[j]);
                return r;
            }
        }
        return KDEFFT_OK;
    }
    KCU(cudaSetDevice(c->device));
    std::vector<std::unique_ptr<kdefft_ds_s>> dss(nds);
    std::vector<BinJob> jobs(nds);
    long long totx = 0, totcells = 0;
    std::vector<long long> xoff(nds, -1), coff(nds);
    int K = 32;
    for (int i = 0; i < nds; ++i) {
        if (n[i] < 1 || !X[i]) return fail(KDEFFT_ERR_ARG, "need n >= 1 samples for every dataset");
        if (o.exact_loo && n[i] < 2) return fail(KDEFFT_ERR_ARG, kLooNeedsTwo);
        dss[i].reset(new kdefft_ds_s());
        kdefft_ds_s& ds = *dss[i];
        ds.ctx = c;
        attach_cache(ds, c);
        ds.d = d;
        ds.n = n[i];
        ds.opts = o;
        BinJob& jb = jobs[i];
        std::memset(&jb, 0, sizeof(jb));
        jb.g.d = d;
        ds.ncells = 1;
        for (int k = 0; k < d; ++k) {
            const double l = lo[(size_t)i * d + k], h = hi[(size_t)i * d + k];
            const int64_t m = M[(size_t)i * d + k];
            if (m < 2 || m > (1 << 20)) return fail(KDEFFT_ERR_ARG, "M_k must be in [2, 2^20]");
            if (!(h > l) || !std::isfinite(l) || !std::isfinite(h)) return fail(KDEFFT_ERR_ARG, "need lo_k < hi_k, finite");
            ds.lo[k] = l;
            ds.hi[k] = h;
            ds.M[k] = m;
            ds.delta[k] = (h - l) / (double)(m - 1);   // Eq. 16
            jb.g.lo[k] = l;
            jb.g.hi[k] = h;
            jb.g.delta[k] = ds.delta[k];
            jb.g.M[k] = m;
            ds.ncells *= m;
        }
        if (ds.ncells > (1LL << 31)) return fail(KDEFFT_ERR_UNSUPPORTED, "grid too large");
        while (K > 8 && (double)n[i] * std::ldexp(1.0, K) >= std::ldexp(1.0, 63)) --K;
        if (!is_device_ptr(X[i])) {
            xoff[i] = totx;
            totx += n[i] * d;
        }
        coff[i] = totcells;
        totcells += (ds.ncells + 3) & ~3LL;   // 16-byte aligned views
        jb.n = n[i];
        jb.ncells = ds.ncells;
        jb.mblk = (int)std::min<long long>(64, (n[i] + 255) / 256);
    }
    // device memory: the samples given on the host, the counts of every
    // dataset (one pool the datasets share), fixed-point accumulators, and
    // outside counters | means | moment partials
    DevBuf xbuf(&c->cache);
    if (totx) KCHK(xbuf.ensure(sizeof(double) * totx));
    auto pool = std::make_shared<DevBuf>(&c->cache);
    KCHK(pool->ensure(sizeof(float) * std::max<long long>(totcells, 1)));
    KCHK(c->binfix.ensure(8 * (size_t)std::max<long long>(totcells, 1)));
    const int nv = d + d * d;
    long long totpart = 0;
    for (int i = 0; i < nds; ++i) totpart += (long long)jobs[i].mblk * nv;
    DevBuf misc(&c->cache);
    const size_t nmisc = (size_t)nds + (size_t)totpart;
    KCHK(misc.ensure(sizeof(double) * nmisc));
    KCU(cudaMemsetAsync(misc.p, 0, sizeof(double) * nds, c->stream));
    KCU(cudaMemsetAsync(c->binfix.p, 0, 8 * (size_t)totcells, c->stream));
    unsigned long long* dOut = (unsigned long long*)misc.p;
    double* dPart = (double*)misc.p + nds;
    KCHK(c->binjobs.ensure(sizeof(BinJob) * nds * 4));
    BinJob* jd = (BinJob*)c->binjobs.p;
    long long po = 0;
    for (int i = 0; i < nds; ++i) {
        BinJob& jb = jobs[i];
        if (xoff[i] >= 0) {
            double* dst = (double*)xbuf.p + xoff[i];
            KCU(cudaMemcpyAsync(dst, X[i], sizeof(double) * n[i] * d, cudaMemcpyHostToDevice, c->stream));
            c->h2d += (int64_t)(sizeof(double) * n[i] * d);
            jb.X = dst;
        } else {
            jb.X = X[i];
        }
        jb.fix = (unsigned long long*)c->binfix.p + coff[i];
        jb.counts = (float*)pool->p + coff[i];
        jb.outside = dOut + i;
        jb.part = dPart + po;
        for (int k = 0; k < d; ++k) jb.shift[k] = 0.5 * (lo[(size_t)i * d + k] + hi[(size_t)i * d + k]);
        po += (long long)jb.mblk * nv;
        dss[i]->pool = pool;
        dss[i]->counts.view(jb.counts, sizeof(float) * (size_t)dss[i]->ncells);
    }
    const double qscale = std::ldexp(1.0, K);
    double by = 0.0, fl = 0.0;
    for (int i = 0; i < nds; ++i) {
        by += (double)n[i] * d * 8.0 + 4.0 * (double)dss[i]->ncells;
        fl += (double)n[i] * (1 << d) * 2.0;
    }
    cudaEvent_t evb = prof_start(c);
    c->launches++;   // phases 0 and 1
    KCU(launch_bin_many(jobs.data(), jd, nds, 0, qscale, c->stream));
    KCU(launch_bin_many(jobs.data(), jd + nds, nds, 1, qscale, c->stream));
    prof_stop(c, evb, "bin", by, fl);
    c->launches += 1;   // the one-pass covariance
    KCU(launch_bin_many(jobs.data(), jd + 2 * nds, nds, 2, qscale, c->stream));
    std::vector<double> part((size_t)totpart);
    std::vector<unsigned long long> nout(nds);
    KCU(cudaMemcpyAsync(nout.data(), dOut, sizeof(unsigned long long) * nds, cudaMemcpyDeviceToHost, c->stream));
    KCU(cudaMemcpyAsync(part.data(), dPart, sizeof(double) * totpart, cudaMemcpyDeviceToHost, c->stream));
    KCU(cudaStreamSynchronize(c->stream));
    prof_flush(c);
    po = 0;
    for (int i = 0; i < nds; ++i) {
        double hs[20] = {0};
        for (int b = 0; b < jobs[i].mblk; ++b)
            for (int v = 0; v < nv; ++v) hs[v] += part[(size_t)(po + (long long)b * nv + v)];
        po += (long long)jobs[i].mblk * nv;
        const double ni = (double)n[i];
        for (int a = 0; a < d; ++a)
            for (int e = 0; e < d; ++e)
                dss[i]->cov[a * d + e] = (n[i] > 1) ? (hs[d + a * d + e] - hs[a] * hs[e] / ni) / (ni - 1.0) : 0.0;
        if (nout[i] > 0 && o.outside_policy == KDEFFT_OUTSIDE_ERROR)
            return fail(KDEFFT_ERR_OUTSIDE_GRID, "dataset " + std::to_string(i) + ": " + std::to_string(nout[i]) +
                                                     " sample points outside the grid");
        dss[i]->dropped = (int64_t)nout[i];
    }
    for (int i = 0; i < nds; ++i) {
        out[i] = dss[i].release();
        c->datasets.push_back(out[i]);
        live_add(out[i]);
    }
    return KDEFFT_OK;
}

int kdefft_ds_destroy(kdefft_ds ds) {
    if (!ds) return KDEFFT_OK;
    if (!live_take(ds)) return fail(KDEFFT_ERR_ARG, "unknown or already destroyed dataset");
    auto& v = ds->ctx->datasets;
    auto it = std::find(v.begin(), v.end(), ds);
    if (it == v.end()) return fail(KDEFFT_ERR_ARG, "unknown or already destroyed dataset");
    v.erase(it);
    ds_free(ds);
    return KDEFFT_OK;
}

int kdefft_ds_set_opts(kdefft_ds ds, const kdefft_opts* o) {
    if (!ds || !o) return fail(KDEFFT_ERR_ARG, "NULL argument");
    if (!(o->tau > 0.0)) return fail(KDEFFT_ERR_ARG, "tau must be positive");
    if (o->exact_loo && ds->n < 2) return fail(KDEFFT_ERR_ARG, kLooNeedsTwo);
    ds->opts.tau = o->tau;
    ds->opts.L_basis = o->L_basis;
    ds->opts.P_rule = o->P_rule;
    std::memcpy(ds->opts.P_fixed, o->P_fixed, sizeof(o->P_fixed));
    ds->opts.exact_loo = o->exact_loo;
    return KDEFFT_OK;
}

int kdefft_ds_info(kdefft_ds ds, int64_t* n, int* d, int64_t* dropped) {
    if (!ds) return fail(KDEFFT_ERR_ARG, "NULL dataset");
    if (n) *n = ds->n;
    if (d) *d = ds->d;
    if (dropped) *dropped = ds->dropped;
    return KDEFFT_OK;
}

int kdefft_counts(kdefft_ds ds, void* dst, int dtype) {
    if (!ds || !dst) return fail(KDEFFT_ERR_ARG, "NULL argument");
    kdefft_ctx c = ds->ctx;
    KCU(cudaSetDevice(c->device));
    const size_t nc = (size_t)ds->ncells;
    const bool dbl = ds->opts.precision == KDEFFT_FP64;
    if (dtype == KDEFFT_DT_I32) {
        if (ds->opts.binning != KDEFFT_BIN_SIMPLE) return fail(KDEFFT_ERR_ARG, "integer counts need SIMPLE binning");
        KCU(cudaMemcpyAsync(dst, ds->counts_i.p, 4 * nc, cudaMemcpyDefault, c->stream));
    } else if ((dtype == KDEFFT_DT_F64) == dbl && (dtype == KDEFFT_DT_F32 || dtype == KDEFFT_DT_F64)) {
        KCU(cudaMemcpyAsync(dst, ds->counts.p, (dbl ? 8 : 4) * nc, cudaMemcpyDefault, c->stream));
    } else if (dtype == KDEFFT_DT_F32 || dtype == KDEFFT_DT_F64) {
        // convert on the host
        std::vector<unsigned char> tmp((dbl ? 8 : 4) * nc);
        KCU(cudaMemcpyAsync(tmp.data(), ds->counts.p, tmp.size(), cudaMemcpyDeviceToHost, c->stream));
        KCU(cudaStreamSynchronize(c->stream));
        std::vector<unsigned char> conv((dtype == KDEFFT_DT_F64 ? 8 : 4) * nc);
        for (size_t i = 0; i < nc; ++i) {
            const double v = dbl ? ((double*)tmp.data())[i] : (double)((float*)tmp.data())[i];
            if (dtype == KDEFFT_DT_F64)
                ((double*)conv.data())[i] = v;
            else
                ((float*)conv.data())[i] = (float)v;
        }
        KCU(cudaMemcpyAsync(dst, conv.data(), conv.size(), cudaMemcpyDefault, c->stream));
    } else {
        return fail(KDEFFT_ERR_ARG, "unknown dtype");
    }
    KCU(cudaStreamSynchronize(c->stream));
    return KDEFFT_OK;
}

int kdefft_plan(kdefft_ds ds, int method, const double* H, const double* G, int* L_out, int* P_out) {
    if (!ds || !H || !L_out || !P_out) return fail(KDEFFT_ERR_ARG, "NULL argument");
    const int d = ds->d;
    Mat Hm, Gm;
    KCHK(sym_check(H, d, Hm, "H"));
    KCHK(spd_or_fail(Hm, "H"));
    Mat basis = Hm;
    if (method == KDEFFT_LSCV) {
        if (ds->opts.L_basis == KDEFFT_L_WIDEST) basis = scaled(2.0, Hm);
    } else if (method == KDEFFT_SCV) {
        if (!G) return fail(KDEFFT_ERR_ARG, "SCV needs G");
        KCHK(sym_check(G, d, Gm, "G"));
        if (ds->opts.L_basis != KDEFFT_L_PAPER) basis = lin(2.0, Hm, 2.0, Gm);
    } else if (method == KDEFFT_PI) {
        if (!G) return fail(KDEFFT_ERR_ARG, "PI needs G");
        KCHK(sym_check(G, d, Gm, "G"));
        basis = Gm;
    }
    return plan_for(ds, basis, L_out, P_out);
}

static int check_common(kdefft_ds ds, const double* H, int nH) {
    if (!ds || !H) return fail(KDEFFT_ERR_ARG, "NULL argument");
    if (nH < 1) return fail(KDEFFT_ERR_ARG, "nH must be >= 1");
    if (cudaSetDevice(ds->ctx->device) != cudaSuccess) return fail(KDEFFT_ERR_CUDA, "cudaSetDevice failed");
    return KDEFFT_OK;
}

int kdefft_psi(kdefft_ds ds, const double* H, int nH, int r, double* out) {
    KCHK(check_common(ds, H, nH));
    HostTimer ht(ds->ctx, "host:psi");
    if (!out) return fail(KDEFFT_ERR_ARG, "NULL output");
    const int d = ds->d;
    if (r < 0 || (r & 1) || r > kRmax[d]) return fail(KDEFFT_ERR_ARG, "r must be even and within the order limit");
    ReqSet rs;
    std::vector<int> first(nH);
    const std::vector<MultiIndex> alphas = order_alphas(d, r);
    {
        HostTimer hq(ds->ctx, "host:psi_requests");
        std::vector<Mat> Hs((size_t)nH);
        for (int h = 0; h < nH; ++h) {
            KCHK(sym_check(H + (size_t)h * d * d, d, Hs[h], "H"));
            KCHK(spd_or_fail(Hs[h], "H"));
        }
        KCHK(add_psi_many(rs, ds, Hs, alphas, first));
    }
    KCHK(run(ds->ctx, rs));
    const std::vector<int> map = kron_map(d, r, alphas);
    const size_t len = map.size();
    std::vector<double> res(len * nH);
    for (int h = 0; h < nH; ++h) kron_expand(map, &rs.grids[first[h]], res.data() + (size_t)h * len);
    return write_out(ds->ctx, out, res.data(), res.size());
}

int kdefft_psi_grad(kdefft_ds ds, const double* H, int nH, int r, const double* w, double* out) {
    KCHK(check_common(ds, H, nH));
    if (!out || !w) return fail(KDEFFT_ERR_ARG, "NULL argument");
    const int d = ds->d;
    if (r < 0 || (r & 1)) return fail(KDEFFT_ERR_ARG, "r must be even");
    if (r + 2 > kRmax[d]) return fail(KDEFFT_ERR_UNSUPPORTED, "the adjoint of psi_r needs psi_{r+2} within the order limit");
    size_t len = 1;
    for (int i = 0; i < r; ++i) len *= (size_t)d;
    // psi_{r+2} at every bandwidth (Kronecker order: position i d^2 + a d + b
    // holds d^{alpha(i) + e_a + e_b} phi), then the contraction with w: the
    // heat equation gives d psi_alpha / d H_ab = 1/2 psi_{alpha + e_a + e_b}
    // for the entries of H taken as independent
    std::vector<double> p2(len * d * d * (size_t)nH);
    KCHK(kdefft_psi(ds, H, nH, r + 2, p2.data()));
    std::vector<double> wh(len * (size_t)nH);
    if (is_device_ptr(w)) {
        KCU(cudaMemcpyAsync(wh.data(), w, sizeof(double) * wh.size(), cudaMemcpyDeviceToHost, ds->ctx->stream));
        KCU(cudaStreamSynchronize(ds->ctx->stream));
        ds->ctx->d2h += (int64_t)(sizeof(double) * wh.size());
    } else {
        std::memcpy(wh.data(), w, sizeof(double) * wh.size());
    }
    std::vector<double> g((size_t)nH * d * d, 0.0);
    for (int h = 0; h < nH; ++h)
        for (size_t i = 0; i < len; ++i) {
            const double wi = 0.5 * wh[(size_t)h * len + i];
            if (wi == 0.0) continue;
            const double* q = &p2[((size_t)h * len + i) * d * d];
            double* gh = &g[(size_t)h * d * d];
            for (int e = 0; e < d * d; ++e) gh[e] += wi * q[e];
        }
    return write_out(ds->ctx, out, g.data(), g.size());
}

// LSCV at nH bandwidths in two halves around run(): the requests, then the
// assembly, so that several criteria can share one run()
struct LscvJob {
    std::vector<int> first;
    std::vector<Mat> Hs;
};

static int lscv_requests(ReqSet& rs, kdefft_ds ds, const double* H, int nH, bool grad, LscvJob& j) {
    const int d = ds->d;
    j.Hs.assign(nH, Mat());
    for (int h = 0; h < nH; ++h) KCHK(sym_check(H + (size_t)h * d * d, d, j.Hs[h], "H"));
    return add_lscv_many(rs, std::vector<kdefft_ds>((size_t)nH, ds), j.Hs, grad, j.first);
}

static void lscv_assemble(const ReqSet& rs, kdefft_ds ds, const LscvJob& j, std::vector<double>& val,
                          std::vector<double>* grad) {
    const int d = ds->d, nH = (int)j.first.size();
    val.assign(nH, 0.0);
    if (grad) grad->assign((size_t)nH * d * d, 0.0);
    for (int h = 0; h < nH; ++h)
        assemble_lscv(ds, j.Hs[h], &rs.grids[j.first[h]], &val[h], grad ? grad->data() + (size_t)h * d * d : nullptr);
}

static int eval_lscv(kdefft_ds ds, const double* H, int nH, std::vector<double>& val, std::vector<double>* grad) {
    ReqSet rs;
    LscvJob j;
    KCHK(lscv_requests(rs, ds, H, nH, grad != nullptr, j));
    KCHK(run(ds->ctx, rs));
    lscv_assemble(rs, ds, j, val, grad);
    return KDEFFT_OK;
}

// n^-2 sum sum phi_{2G}(X_i - X_j) at truncation L and padding P: the
// H-independent SCV term, cached per dataset
static std::vector<double> c2g_key(const Mat& G, const int* L, const int* P, int d) {
    std::vector<double> k;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) k.push_back(G(a, b));
    for (int i = 0; i < d; ++i) {
        k.push_back(L[i]);
        k.push_back(P[i]);
    }
    return k;
}

// SCV at nH bandwidths in the same two halves (the phi_2G sums missing from
// the dataset's cache are requested too, and cached by the assembly)
struct ScvJob {
    std::vector<int> first;
    std::vector<Mat> Hs;
    std::vector<std::vector<double>> keys;
    std::map<std::vector<double>, int> missing;   // key -> grid index of its phi_2G request
    bool split64 = true;
};

static int scv_requests(ReqSet& rs, kdefft_ds ds, const double* H, int nH, const Mat& G, bool grad, bool split64,
                        ScvJob& j) {
    const int d = ds->d;
    j.first.assign(nH, 0);
    j.Hs.assign(nH, Mat());
    j.keys.assign(nH, {});
    j.missing.clear();
    j.split64 = split64;
    std::vector<int>& first = j.first;
    std::vector<Mat>& Hs = j.Hs;
    std::vector<std::vector<double>>& keys = j.keys;
    std::map<std::vector<double>, int>& missing = j.missing;
    for (int h = 0; h < nH; ++h) {
        KCHK(sym_check(H + (size_t)h * d * d, d, Hs[h], "H"));
        KCHK(add_scv(rs, ds, Hs[h], G, grad, split64, first[h]));
        const GridReq& g0 = rs.grids[first[h]];
        keys[h] = c2g_key(G, g0.L, g0.P, d);
        if (split64 && !ds->c2g.count(keys[h]) && !missing.count(keys[h])) {
            KSpec sp;
            sp.nsig = 1;
            sp.sig[0] = scaled(2.0, G);
            const int si = (int)rs.specs.size();
            rs.specs.push_back(sp);
            GridReq g;
            g.ds = ds;
            g.spec = si;
            std::memcpy(g.L, g0.L, sizeof(g.L));
            std::memcpy(g.P, g0.P, sizeof(g.P));
            g.terms = {Term{0, {0}, 1.0}};
            g.fp64 = true;
            missing[keys[h]] = (int)rs.grids.size();
            rs.grids.push_back(std::move(g));
        }
    }
    return KDEFFT_OK;
}

static void scv_assemble(const ReqSet& rs, kdefft_ds ds, const ScvJob& j, std::vector<double>& val,
                         std::vector<double>* grad) {
    const int d = ds->d, nH = (int)j.first.size();
    for (const auto& kv : j.missing) ds->c2g[kv.first] = rs.grids[kv.second].value;
    val.assign(nH, 0.0);
    if (grad) grad->assign((size_t)nH * d * d, 0.0);
    for (int h = 0; h < nH; ++h)
        assemble_scv(ds, j.Hs[h], &rs.grids[j.first[h]], j.split64, j.split64 ? ds->c2g[j.keys[h]] : 0.0, &val[h],
                     grad ? grad->data() + (size_t)h * d * d : nullptr);
}

static int eval_scv(kdefft_ds ds, const double* H, int nH, const Mat& G, std::vector<double>& val,
                    std::vector<double>* grad, bool split64 = true) {
    ReqSet rs;
    ScvJob j;
    KCHK(scv_requests(rs, ds, H, nH, G, grad != nullptr, split64, j));
    KCHK(run(ds->ctx, rs));
    scv_assemble(rs, ds, j, val, grad);
    return KDEFFT_OK;
}

static int psi4_kron(kdefft_ds ds, const Mat& G, std::vector<double>& psi4) {
    const int d = ds->d;
    ReqSet rs;
    int first;
    const std::vector<MultiIndex> alphas = order_alphas(d, 4);
    KCHK(spd_or_fail(G, "G"));
    KCHK(add_psi(rs, ds, G, alphas, first));
    KCHK(run(ds->ctx, rs));
    psi4.assign((size_t)d * d * d * d, 0.0);
    kron_expand(kron_map(d, 4, alphas), &rs.grids[first], psi4.data());
    return KDEFFT_OK;
}

static int eval_pi(kdefft_ds ds, const double* H, int nH, const std::vector<double>& psi4, std::vector<double>& val,
                   std::vector<double>* grad) {
    const int d = ds->d;
    val.assign(nH, 0.0);
    if (grad) grad->assign((size_t)nH * d * d, 0.0);
    for (int h = 0; h < nH; ++h) {
        Mat Hm;
        KCHK(sym_check(H + (size_t)h * d * d, d, Hm, "H"));
        KCHK(spd_or_fail(Hm, "H"));
        assemble_pi(ds, Hm, psi4.data(), &val[h], grad ? grad->data() + (size_t)h * d * d : nullptr);
    }
    return KDEFFT_OK;
}

static int get_G(kdefft_ds ds, const double* G, Mat& Gm) {
    const int d = ds->d;
    if (G) {
        KCHK(sym_check(G, d, Gm, "G"));
        KCHK(spd_or_fail(Gm, "G"));
    } else {
        // normal-scale matrix (4/(d+2))^{2/(d+4)} n^{-2/(d+4)} S
        const double f = std::pow(4.0 / (d + 2.0), 2.0 / (d + 4.0)) * std::pow((double)ds->n, -2.0 / (d + 4.0));
        Gm = Mat();
        Gm.d = d;
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) Gm(a, b) = f * ds->cov[a * d + b];
    }
    return spd_or_fail(Gm, "G");
}

int kdefft_lscv(kdefft_ds ds, const double* H, int nH, double* val, double* grad) {
    KCHK(check_common(ds, H, nH));
    if (!val) return fail(KDEFFT_ERR_ARG, "NULL output");
    std::vector<double> v, g;
    KCHK(eval_lscv(ds, H, nH, v, grad ? &g : nullptr));
    KCHK(write_out(ds->ctx, val, v.data(), v.size()));
    if (grad) KCHK(write_out(ds->ctx, grad, g.data(), g.size()));
    return KDEFFT_OK;
}

int kdefft_scv(kdefft_ds ds, const double* H, int nH, const double* G, double* val, double* grad) {
    KCHK(check_common(ds, H, nH));
    if (!val || !G) return fail(KDEFFT_ERR_ARG, "NULL argument");
    Mat Gm;
    KCHK(get_G(ds, G, Gm));
    std::vector<double> v, g;
    KCHK(eval_scv(ds, H, nH, Gm, v, grad ? &g : nullptr));
    KCHK(write_out(ds->ctx, val, v.data(), v.size()));
    if (grad) KCHK(write_out(ds->ctx, grad, g.data(), g.size()));
    return KDEFFT_OK;
}

int kdefft_pi(kdefft_ds ds, const double* H, int nH, const double* G, double* val, double* grad) {
    KCHK(check_common(ds, H, nH));
    if (!val || !G) return fail(KDEFFT_ERR_ARG, "NULL argument");
    Mat Gm;
    KCHK(get_G(ds, G, Gm));
    std::vector<double> psi4, v, g;
    KCHK(psi4_kron(ds, Gm, psi4));
    KCHK(eval_pi(ds, H, nH, psi4, v, grad ? &g : nullptr));
    KCHK(write_out(ds->ctx, val, v.data(), v.size()));
    if (grad) KCHK(write_out(ds->ctx, grad, g.data(), g.size()));
    return KDEFFT_OK;
}

int kdefft_eta02(kdefft_ds ds, const double* H, int nH, const double* G, double* val) {
    KCHK(check_common(ds, H, nH));
    if (!val || !G) return fail(KDEFFT_ERR_ARG, "NULL argument");
    const int d = ds->d;
    if (kRmax[d] < 4) return fail(KDEFFT_ERR_UNSUPPORTED, "order 4 not available");
    Mat Gm;
    KCHK(get_G(ds, G, Gm));
    ReqSet rs;
    std::vector<int> first(nH);
    for (int h = 0; h < nH; ++h) {
        Mat Hm;
        KCHK(sym_check(H + (size_t)h * d * d, d, Hm, "H"));
        KCHK(add_eta02(rs, ds, Hm, Gm, first[h]));
    }
    KCHK(run(ds->ctx, rs));
    std::vector<double> v(nH);
    for (int h = 0; h < nH; ++h) v[h] = rs.grids[first[h]].value;
    return write_out(ds->ctx, val, v.data(), v.size());
}

int kdefft_qr(kdefft_ds ds, const double* Sigma, int nS, int r, double* out) {
    KCHK(check_common(ds, Sigma, nS));
    if (!out) return fail(KDEFFT_ERR_ARG, "NULL output");
    const int d = ds->d;
    if (r < 0 || (r & 1) || r > kRmax[d]) return fail(KDEFFT_ERR_ARG, "r must be even and within the order limit");
    ReqSet rs;
    std::vector<int> first(nS);
    for (int i = 0; i < nS; ++i) {
        Mat Sg;
        KCHK(sym_check(Sigma + (size_t)i * d * d, d, Sg, "Sigma"));
        KCHK(add_eta_m(rs, ds, Sg, r / 2, first[i]));
    }
    KCHK(run(ds->ctx, rs));
    std::vector<double> v(nS);
    for (int i = 0; i < nS; ++i) v[i] = rs.grids[first[i]].value;
    return write_out(ds->ctx, out, v.data(), v.size());
}

int kdefft_eta_rs(kdefft_ds ds, const double* A, const double* B, const double* Sigma, int nS, int r, int s,
                  double* out) {
    KCHK(check_common(ds, Sigma, nS));
    if (!out) return fail(KDEFFT_ERR_ARG, "NULL output");
    const int d = ds->d;
    if (r < 0 || s < 0 || 2 * (r + s) > kRmax[d]) return fail(KDEFFT_ERR_ARG, "2(r + s) must be within the order limit");
    Mat Am, Bm;
    Am.d = Bm.d = d;
    for (int i = 0; i < d; ++i) Am(i, i) = Bm(i, i) = 1.0;
    if (A) KCHK(sym_check(A, d, Am, "A"));
    if (B) KCHK(sym_check(B, d, Bm, "B"));
    ReqSet rs;
    std::vector<int> first(nS);
    for (int i = 0; i < nS; ++i) {
        Mat Sg;
        KCHK(sym_check(Sigma + (size_t)i * d * d, d, Sg, "Sigma"));
        KCHK(add_eta_rs(rs, ds, Am, Bm, Sg, r, s, first[i]));
    }
    KCHK(run(ds->ctx, rs));
    std::vector<double> v(nS);
    for (int i = 0; i < nS; ++i) v[i] = rs.grids[first[i]].value;
    return write_out(ds->ctx, out, v.data(), v.size());
}

static KdeDesc kde_desc(kdefft_ds ds, const int* L) {
    KdeDesc g;
    std::memset(&g, 0, sizeof(g));
    g.d = ds->d;
    g.ncells = ds->ncells;
    g.nstencil = 1;
    for (int k = 0; k < ds->d; ++k) {
        g.M[k] = ds->M[k];
        g.L[k] = L ? L[k] : 0;
        g.nstencil *= 2 * g.L[k] + 1;
        g.lo[k] = ds->lo[k];
        g.delta[k] = ds->delta[k];
    }
    g.inv_n = 1.0 / (double)ds->n;
    return g;
}

int kdefft_kde_grid(kdefft_ds ds, const double* H, double* out) {
    KCHK(check_common(ds, H, 1));
    if (!out) return fail(KDEFFT_ERR_ARG, "NULL output");
    if (ds->opts.precision != KDEFFT_FP32 || ds->opts.binning != KDEFFT_BIN_LINEAR)
        return fail(KDEFFT_ERR_UNSUPPORTED, "the grid estimate takes FP32 linear-binned datasets");
    kdefft_ctx c = ds->ctx;
    const int d = ds->d;
    Mat Hm;
    KCHK(sym_check(H, d, Hm, "H"));
    KCHK(spd_or_fail(Hm, "H"));
    int L[4] = {0, 0, 0, 0}, P[4];
    KCHK(plan_for(ds, Hm, L, P));
    const KdeDesc g = kde_desc(ds, L);
    // stencil K_H(delta (.) l), last axis fastest, FP64 on the host
    Mat inv;
    double det;
    spd_inv_det(Hm, inv, det);
    const double nrm = std::pow(2.0 * M_PI, -0.5 * d) / std::sqrt(det);
    std::vector<float> tab((size_t)g.nstencil);
    for (long long s = 0; s < g.nstencil; ++s) {
        long long r = s;
        double x[4] = {0, 0, 0, 0};
        for (int k = d - 1; k >= 0; --k) {
            const int w = 2 * L[k] + 1;
            x[k] = ds->delta[k] * (double)((int)(r % w) - L[k]);
            r /= w;
        }
        double q = 0.0;
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) q += x[a] * inv(a, b) * x[b];
        tab[(size_t)s] = (float)(nrm * std::exp(-0.5 * q));
    }
    const size_t bt = (sizeof(float) * tab.size() + 255) & ~(size_t)255;
    KCHK(c->kdebuf.ensure(bt + sizeof(double) * (size_t)ds->ncells));
    float* dtab = (float*)c->kdebuf.p;
    double* dout = (double*)((unsigned char*)c->kdebuf.p + bt);
    KCU(cudaMemcpyAsync(dtab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice, c->stream));
    c->h2d += (int64_t)(sizeof(float) * tab.size());
    cudaEvent_t ev = prof_start(c);
    KCU(launch_kde_grid((const float*)ds->counts.p, g, dtab, dout, c->nsm, c->stream));
    prof_stop(c, ev, "kde_grid", 8.0 * (double)ds->ncells + 4.0 * (double)g.nstencil,
              2.0 * (double)ds->ncells * (double)g.nstencil);
    if (is_device_ptr(out)) {
        KCU(cudaMemcpyAsync(out, dout, sizeof(double) * ds->ncells, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        KCU(cudaMemcpyAsync(out, dout, sizeof(double) * ds->ncells, cudaMemcpyDeviceToHost, c->stream));
        c->d2h += (int64_t)(sizeof(double) * ds->ncells);
    }
    KCU(cudaStreamSynchronize(c->stream));
    prof_flush(c);
    return KDEFFT_OK;
}

int kdefft_ise_mixture(kdefft_ds ds, const double* H, int nH, int K, const double* w, const double* mu,
                       const double* S, double* out) {
    KCHK(check_common(ds, H, nH));
    if (!out || !w || !mu || !S || K < 1 || K > 64) return fail(KDEFFT_ERR_ARG, "need 1..64 mixture components");
    if (ds->opts.precision != KDEFFT_FP32 || ds->opts.binning != KDEFFT_BIN_LINEAR)
        return fail(KDEFFT_ERR_UNSUPPORTED, "the mixture ISE takes FP32 linear-binned datasets");
    kdefft_ctx c = ds->ctx;
    const int d = ds->d;
    std::vector<Mat> Sm(K);
    for (int m = 0; m < K; ++m) {
        KCHK(sym_check(S + (size_t)m * d * d, d, Sm[m], "mixture covariance"));
        KCHK(spd_or_fail(Sm[m], "mixture covariance"));
    }
    auto gauss_at = [&](const Mat& Sg, const double* x) {   // phi_Sg(x), FP64
        Mat inv;
        double det;
        spd_inv_det(Sg, inv, det);
        double q = 0.0;
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) q += x[a] * inv(a, b) * x[b];
        return std::pow(2.0 * M_PI, -0.5 * d) / std::sqrt(det) * std::exp(-0.5 * q);
    };
    // int f^2 = sum_lm w_l w_m phi_{S_l + S_m}(mu_l - mu_m), closed form
    double ff = 0.0;
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b) {
            double x[4];
            for (int k = 0; k < d; ++k) x[k] = mu[(size_t)a * d + k] - mu[(size_t)b * d + k];
            ff += w[a] * w[b] * gauss_at(lin(1.0, Sm[a], 1.0, Sm[b]), x);
        }
    // int f_hat^2 = n^-2 sum_ij phi_2H (binned, the lag-domain or FFT engine)
    ReqSet rs;
    std::vector<int> first(nH);
    std::vector<Mat> Hs(nH);
    for (int h = 0; h < nH; ++h) {
        KCHK(sym_check(H + (size_t)h * d * d, d, Hs[h], "H"));
        KCHK(add_eta_m(rs, ds, scaled(2.0, Hs[h]), 0, first[h]));
    }
    KCHK(run(c, rs));
    // int f_hat f = n^-1 sum_g c_g sum_m w_m phi_{H + S_m}(x_g - mu_m)
    const KdeDesc g = kde_desc(ds, nullptr);
    const int nb = std::max(1, std::min(c->nsm * 4, (int)((ds->ncells + 255) / 256)));
    const size_t bc = (sizeof(MixComp) * K + 255) & ~(size_t)255;
    KCHK(c->kdebuf.ensure(bc + sizeof(double) * nb));
    MixComp* dcomp = (MixComp*)c->kdebuf.p;
    double* dpart = (double*)((unsigned char*)c->kdebuf.p + bc);
    std::vector<double> v(nH), part(nb);
    for (int h = 0; h < nH; ++h) {
        std::vector<MixComp> comps(K);
        for (int m = 0; m < K; ++m) {
            std::memset(&comps[m], 0, sizeof(MixComp));
            const Mat Sc = lin(1.0, Hs[h], 1.0, Sm[m]);
            Mat inv;
            double det;
            spd_inv_det(Sc, inv, det);
            for (int k = 0; k < d; ++k) comps[m].mu[k] = mu[(size_t)m * d + k];
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) comps[m].lam[a * MAXD + b] = inv(a, b);
            comps[m].nrm = std::pow(2.0 * M_PI, -0.5 * d) / std::sqrt(det);
            comps[m].w = w[m];
        }
        KCU(cudaMemcpyAsync(dcomp, comps.data(), sizeof(MixComp) * K, cudaMemcpyHostToDevice, c->stream));
        cudaEvent_t ev = prof_start(c);
        KCU(launch_mix_dot((const float*)ds->counts.p, g, dcomp, K, dpart, nb, c->stream));
        prof_stop(c, ev, "mix_dot", 4.0 * (double)ds->ncells, 12.0 * (double)ds->ncells * K);
        KCU(cudaMemcpyAsync(part.data(), dpart, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream));
        KCU(cudaStreamSynchronize(c->stream));
        double cross = 0.0;
        for (int b = 0; b < nb; ++b) cross += part[b];
        cross /= (double)ds->n;
        v[h] = rs.grids[first[h]].value - 2.0 * cross + ff;
    }
    prof_flush(c);
    return write_out(c, out, v.data(), v.size());
}

int kdefft_lscv_r(kdefft_ds ds, const double* H, int nH, int r, double* val) {
    KCHK(check_common(ds, H, nH));
    if (!val) return fail(KDEFFT_ERR_ARG, "NULL output");
    const int d = ds->d;
    if (r < 0 || 2 * r > kRmax[d]) return fail(KDEFFT_ERR_ARG, "2r must be within the order limit");
    ReqSet rs;
    std::vector<int> first(nH);
    std::vector<Mat> Hs(nH);
    for (int h = 0; h < nH; ++h) {
        KCHK(sym_check(H + (size_t)h * d * d, d, Hs[h], "H"));
        KCHK(add_lscv_r(rs, ds, Hs[h], r, first[h]));
    }
    KCHK(run(ds->ctx, rs));
    const double n = (double)ds->n;
    const double sgn = (r & 1) ? -1.0 : 1.0;
    std::vector<double> v(nH);
    for (int h = 0; h < nH; ++h) {
        // eta_r(0; H) = sum_beta r!/beta! d^{2 beta} phi_H(0)
        std::vector<Term> t0;
        laplacian_power_terms(d, r, 0, 1.0, t0);
        double e0 = 0.0;
        for (const Term& t : t0) e0 += t.w * dphi_at0(Hs[h], t.alpha);
        if (!ds->opts.exact_loo) {
            v[h] = sgn * (rs.grids[first[h]].value + 2.0 * e0 / n);   // Eq. 36
        } else {
            const double A = rs.grids[first[h]].value, B = rs.grids[first[h] + 1].value;
            v[h] = sgn * (A - 2.0 / (n * (n - 1.0)) * (n * n * B - n * e0));   // Eq. 35
        }
    }
    return write_out(ds->ctx, val, v.data(), v.size());
}

int kdefft_batch_lscv(kdefft_ctx c, int nds, const kdefft_ds* dss, const int* nH_per_ds, const double* H,
                      double* val, double* grad) {
    if (!c || !dss || !nH_per_ds || !H || !val || nds < 1) return fail(KDEFFT_ERR_ARG, "NULL argument");
    KCU(cudaSetDevice(c->device));
    const int d = dss[0]->d;
    const int prec = dss[0]->opts.precision;
    ReqSet rs;
    std::vector<int> first;
    std::vector<Mat> Hs;
    std::vector<kdefft_ds> owner;
    size_t off = 0;
    for (int i = 0; i < nds; ++i) {
        kdefft_ds ds = dss[i];
        if (!ds || ds->ctx != c || ds->d != d || ds->opts.precision != prec)
            return fail(KDEFFT_ERR_ARG, "datasets must share context, d and precision");
        for (int h = 0; h < nH_per_ds[i]; ++h) {
            Mat Hm;
            KCHK(sym_check(H + (off + h) * d * d, d, Hm, "H"));
            Hs.push_back(Hm);
            owner.push_back(ds);
        }
        off += nH_per_ds[i];
    }
    KCHK(add_lscv_many(rs, owner, Hs, grad != nullptr, first));
    KCHK(run(c, rs));
    const size_t nt = Hs.size();
    std::vector<double> v(nt), g(grad ? nt * d * d : 0);
    host_parallel_for(nt, 2048, [&](size_t h0, size_t h1) {
        for (size_t h = h0; h < h1; ++h)
            assemble_lscv(owner[h], Hs[h], &rs.grids[first[h]], &v[h], grad ? g.data() + h * d * d : nullptr);
    });
    std::memcpy(val, v.data(), sizeof(double) * nt);
    if (grad) std::memcpy(grad, g.data(), sizeof(double) * g.size());
    return KDEFFT_OK;
}

}  // extern "C"

// ============================================================ optimiser
// Parametrisation theta: H = R R^T with R lower triangular, R_ii = exp(theta),
// off-diagonal entries free; row-major over the lower triangle.
namespace {

// Search parameters theta of a bandwidth class (Sec. 3): F, the full SPD
// matrices, through the Cholesky factor R (H = R R^T, log diagonal, p =
// d(d+1)/2); D, the diagonal ones, H = diag(e^{2 theta_k}) (p = d); S, the
// scalar ones, H = e^{2 theta} I (p = 1).
struct Opt {
    int d;
    int p;
    int cls = KDEFFT_H_FULL;
};

static int class_params(int d, int cls) { return cls == KDEFFT_H_FULL ? d * (d + 1) / 2 : (cls == KDEFFT_H_DIAG ? d : 1); }

Mat theta_to_H(const Opt& o, const double* th, Mat* Rout = nullptr) {
    Mat R;
    R.d = o.d;
    if (o.cls == KDEFFT_H_DIAG || o.cls == KDEFFT_H_SCALAR) {
        for (int i = 0; i < o.d; ++i) R(i, i) = std::exp(o.cls == KDEFFT_H_DIAG ? th[i] : th[0]);
    } else {
        int t = 0;
        for (int i = 0; i < o.d; ++i)
            for (int j = 0; j <= i; ++j) {
                R(i, j) = (i == j) ? std::exp(th[t]) : th[t];
                ++t;
            }
    }
    Mat H;
    H.d = o.d;
    for (int i = 0; i < o.d; ++i)
        for (int j = 0; j < o.d; ++j) {
            double s = 0.0;
            for (int k = 0; k <= std::min(i, j); ++k) s += R(i, k) * R(j, k);
            H(i, j) = s;
        }
    if (Rout) *Rout = R;
    return H;
}

void H_to_theta(const Opt& o, const Mat& H, double* th) {
    if (o.cls == KDEFFT_H_DIAG) {   // the diagonal of H (the start projected onto D)
        for (int i = 0; i < o.d; ++i) th[i] = 0.5 * std::log(H(i, i));
        return;
    }
    if (o.cls == KDEFFT_H_SCALAR) {   // h^2 = geometric mean of the diagonal
        double s = 0.0;
        for (int i = 0; i < o.d; ++i) s += std::log(H(i, i));
        th[0] = 0.5 * s / o.d;
        return;
    }
    Mat R;
    cholesky(H, R);
    int t = 0;
    for (int i = 0; i < o.d; ++i)
        for (int j = 0; j <= i; ++j) {
            th[t] = (i == j) ? std::log(R(i, i)) : R(i, j);
            ++t;
        }
}

// tied gradient g (d x d) of F(H) -> gradient in theta
void grad_theta(const Opt& o, const double* th, const double* g, double* gt) {
    Mat R;
    const Mat H = theta_to_H(o, th, &R);
    const int d = o.d;
    if (o.cls == KDEFFT_H_DIAG) {   // dH_kk / dtheta_k = 2 H_kk
        for (int k = 0; k < d; ++k) gt[k] = 2.0 * H(k, k) * g[k * d + k];
        return;
    }
    if (o.cls == KDEFFT_H_SCALAR) {   // dH / dtheta = 2 h^2 I
        double tr = 0.0;
        for (int k = 0; k < d; ++k) tr += g[k * d + k];
        gt[0] = 2.0 * H(0, 0) * tr;
        return;
    }
    // independent-entry derivative G_ind: off-diagonals are half the tied values
    Mat Gi;
    Gi.d = d;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) Gi(a, b) = (a == b) ? g[a * d + b] : 0.5 * g[a * d + b];
    // dF/dR = 2 G_ind R
    int t = 0;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += Gi(i, k) * R(k, j);
            s *= 2.0;
            gt[t] = (i == j) ? s * R(i, i) : s;
            ++t;
        }
}

}  // namespace

// FP32 copies of the search parameters (rounded once here, not per round)
static void params_f32(SelectParams& q) {
    q.tauf = (float)q.tau;
    q.d0f = (float)q.delta0;
    q.d1f = (float)q.delta1;
    q.rd0f = 1.0f / q.d0f;   // an IEEE FP32 division: the correctly rounded reciprocal
    q.rd1f = 1.0f / q.d1f;
    for (int e = 0; e < 4; ++e) q.Gf[e] = (float)q.G[e];
    // the pilot's Gaussian phi_{2G}, the base of the SCV kernel's
    // cancellation-free form (zero for LSCV, whose G is zero)
    const double g00 = 2.0 * q.G[0], g01 = 2.0 * 0.5 * (q.G[1] + q.G[2]), g11 = 2.0 * q.G[3];
    const double det = g00 * g11 - g01 * g01;
    const double d0 = q.delta0, d1 = q.delta1;
    auto pair = [](double v, float& h, float& l) {
        h = (float)v;
        l = (float)(v - (double)h);
    };
    const double L[3] = {det > 0.0 ? g11 / det : 0.0, det > 0.0 ? -g01 / det : 0.0, det > 0.0 ? g00 / det : 0.0};
    const double dd[3] = {d0 * d0, d0 * d1, d1 * d1};
    for (int e = 0; e < 3; ++e) {
        pair(L[e], q.l2gh[e], q.l2gl[e]);
        pair(dd[e], q.ddh[e], q.ddl[e]);
        q.l2gj[e] = (float)(dd[e] * L[e]);
        q.gsc[e] = (float)(1.0 / dd[e]);
    }
    pair(det > 0.0 ? 1.0 / det : 0.0, q.dl2gh, q.dl2gl);
    q.n2g = det > 0.0 ? (float)(1.0 / (2.0 * M_PI * std::sqrt(det))) : 0.f;
}

// Whether the device-resident search covers a criterion on this dataset:
// d = 2, FP32, minimal padding, LSCV of Eq. 10 or SCV.
static bool select2d_covered(kdefft_ds ds, int method) {
    kdefft_ctx c = ds->ctx;
    return c->device_select && ds->d == 2 && ds->opts.precision == KDEFFT_FP32 &&
           ds->opts.P_rule == KDEFFT_P_MINIMAL && ds->opts.L_basis != KDEFFT_L_FULL &&
           !(method == KDEFFT_LSCV && ds->opts.exact_loo) && !(method == KDEFFT_SCV && ds->opts.L_basis == KDEFFT_L_PAPER) &&
           (method == KDEFFT_LSCV || method == KDEFFT_SCV);
}

// The lag-domain device search for one or two criteria on one dataset in one
// launch, one CTA per start.  The autocorrelation box covers 2.5 times the
// largest support among all starts of all criteria (the bandwidth may grow
// about 6-fold beyond the widest start); trial points needing more are
// outside the search's domain.
static int device_select2d_lag(kdefft_ds ds, const std::vector<int>& methods, const std::vector<Mat>& Gms,
                               const std::vector<std::vector<std::vector<double>>>& th0s, int max_iter,
                               std::vector<std::vector<std::vector<double>>>& th_outs,
                               std::vector<std::vector<double>>& f_outs, std::vector<int64_t>& evals_out) {
    kdefft_ctx c = ds->ctx;
    const int nm = (int)methods.size();
    if (nm < 1 || nm > 2) return KDEFFT_ERR_UNSUPPORTED;
    const Opt o{2, 3};
    int Lmax[2] = {1, 1};
    for (int m = 0; m < nm; ++m)
        for (const auto& th : th0s[m]) {
            const Mat H = theta_to_H(o, th.data());
            double B[4];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    const double h = H(a, b);
                    if (methods[m] == KDEFFT_SCV)
                        B[a * 2 + b] = 2.0 * h + 2.0 * Gms[m](a, b);
                    else
                        B[a * 2 + b] = (ds->opts.L_basis == KDEFFT_L_WIDEST ? 2.0 : 1.0) * h;
                }
            const double tr = 0.5 * (B[0] + B[3]), dd = 0.5 * (B[0] - B[3]);
            const double lam = tr + std::sqrt(dd * dd + B[1] * B[1]);
            for (int k = 0; k < 2; ++k) {
                double v = std::ceil(ds->opts.tau * std::sqrt(std::fabs(lam)) / ds->delta[k]);
                if (!(v <= (double)(ds->M[k] - 1))) v = (double)(ds->M[k] - 1);
                Lmax[k] = std::max(Lmax[k], (int)std::max(1.0, v));
            }
        }
    std::array<int, 4> need{0, 0, 0, 0};
    for (int k = 0; k < 2; ++k)
        need[k] = (int)std::min<long long>(ds->M[k] - 1, std::max(8, (int)std::ceil(2.5 * Lmax[k])));
    std::vector<int> first(nm + 1, 0);
    for (int m = 0; m < nm; ++m) first[m + 1] = first[m] + (int)th0s[m].size();
    const int nst = first[nm];
    const size_t bT = sizeof(SelStart) * nst;
    KCHK(c->sel_buf.ensure(bT));
    // pinned start table: copied up when the launch sequence runs, and the
    // results come back into it (free again after the synchronisation at
    // the end of every search)
    KCHK(c->h_sel.ensure(bT));
    SelStart* st = (SelStart*)c->h_sel.p;
    for (int m = 0; m < nm; ++m)
        for (int i = 0; i < (int)th0s[m].size(); ++i) {
            SelStart& x = st[first[m] + i];
            std::memset(&x, 0, sizeof(SelStart));
            for (int k = 0; k < 3; ++k) x.th[k] = th0s[m][i][k];
        }
    SelStart* dst = (SelStart*)c->sel_buf.p;
    if (c->rec && (int64_t)nst * c->rec_cap * SEL_REC > c->rec_len)
        return fail(KDEFFT_ERR_ARG, "search record buffer smaller than starts x cap x fields");
    SelectParams prm[2]{};
    cudaEvent_t ev = nullptr;
    // the search's parameters need the final autocorrelation box: set up
    // when the box is (the start table copy, the search and the copy back
    // join the autocorrelation passes' launch sequence)
    StreamTail tail;
    tail.prepare = [&](std::vector<long long>& sig) -> int {
        std::memset(prm, 0, sizeof(prm));   // padding too: the bytes are the signature
        for (int m = 0; m < nm; ++m) {
            SelectParams& q = prm[m];
            const int method = methods[m];
            q.method = (method == KDEFFT_LSCV) ? 0 : 1;
            q.max_iter = max_iter;
            q.widest = (method == KDEFFT_LSCV && ds->opts.L_basis == KDEFFT_L_WIDEST) ? 1 : 0;
            q.M0 = (int)ds->M[0];
            q.M1 = (int)ds->M[1];
            q.Lcap = ds->acA[0];
            q.Lcap1 = ds->acA[1];
            q.n = (double)ds->n;
            q.inv_n = 1.0 / q.n;
            q.inv_n2 = 1.0 / (q.n * q.n);
            q.inv_nf = (float)q.inv_n;
            q.inv_n2h = (float)q.inv_n2;
            q.inv_n2l = (float)(q.inv_n2 - (double)q.inv_n2h);
            q.tau = ds->opts.tau;
            q.delta0 = ds->delta[0];
            q.delta1 = ds->delta[1];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) q.G[a * 2 + b] = (method == KDEFFT_SCV) ? Gms[m](a, b) : 0.0;
            params_f32(q);
            q.errflag = c->errflag;
            q.acorr = (const float*)ds->ac32.p;
            q.A0 = ds->acA[0];
            q.A1 = ds->acA[1];
            q.rec = c->rec;
            q.rec_cap = c->rec_cap;
        }
        if (nm == 1) prm[1] = prm[0];
        // the parameters by value, as the launch captures them
        const size_t w = (sizeof(prm) + sizeof(long long) - 1) / sizeof(long long);
        std::vector<long long> pb(w, 0);
        std::memcpy(pb.data(), prm, sizeof(prm));
        sig.insert(sig.end(), {8, (long long)(uintptr_t)dst, (long long)(uintptr_t)st, (long long)bT, nst, first[1]});
        sig.insert(sig.end(), pb.begin(), pb.end());
        return KDEFFT_OK;
    };
    tail.issue = [&]() -> int {
        KCU(cudaMemcpyAsync(dst, st, bT, cudaMemcpyHostToDevice, c->stream));
        ev = prof_start(c);
        KCU(launch_select2d_lag(prm[0], prm[1], first[1], dst, nst, c->stream));
        prof_stop(c, ev, "select2d_lag_f32", 0.0, 0.0);
        KCU(cudaMemcpyAsync(st, dst, bT, cudaMemcpyDeviceToHost, c->stream));
        return KDEFFT_OK;
    };
    const int ar = ensure_autocorr_many(c, {{ds, need}}, &tail);
    if (ar == KDEFFT_ERR_UNSUPPORTED) return KDEFFT_ERR_UNSUPPORTED;
    KCHK(ar);
    c->h2d += (int64_t)bT;
    {
        HostTimer w(c, "host:wait");
        KCU(cudaStreamSynchronize(c->stream));
    }
    c->d2h += (int64_t)bT;
    if (c->prof && !c->pending.empty() && ev) {
        double fl = 0.0, by = 0.0;
        for (int i = 0; i < nst; ++i) {
            fl += st[i].flops;
            by += st[i].bytes;
        }
        c->pending.back().flops = fl;
        c->pending.back().bytes = by;
    }
    prof_flush(c);
    // (k_select2d_lag has no bounded waits, so it never raises the error flag)
    th_outs.assign(nm, {});
    f_outs.assign(nm, {});
    evals_out.assign(nm, 0);
    for (int m = 0; m < nm; ++m) {
        const int k = first[m + 1] - first[m];
        th_outs[m].assign(k, std::vector<double>(3));
        f_outs[m].assign(k, INFINITY);
        for (int i = 0; i < k; ++i) {
            const SelStart& x = st[first[m] + i];
            for (int e = 0; e < 3; ++e) th_outs[m][i][e] = x.th[e];
            f_outs[m][i] = x.f;
            evals_out[m] += x.evals;
        }
    }
    return KDEFFT_OK;
}

// Device-resident selection for d = 2 (FP32 dataset, LSCV of Eq. 10 or SCV,
// minimal padding): returns KDEFFT_ERR_UNSUPPORTED without side effects when
// the case is not covered, so that the caller runs the host optimiser.
static int device_select2d(kdefft_ds ds, int method, const Mat& Gm, const std::vector<std::vector<double>>& th0,
                           int max_iter, std::vector<std::vector<double>>& th_out, std::vector<double>& f_out,
                           int64_t* evals_out) {
    kdefft_ctx c = ds->ctx;
    if (!select2d_covered(ds, method)) return KDEFFT_ERR_UNSUPPORTED;
    const int nst = (int)th0.size();
    const int M0 = (int)ds->M[0], M1 = (int)ds->M[1];
    if (c->lag) {
        std::vector<std::vector<std::vector<double>>> tho;
        std::vector<std::vector<double>> fo;
        std::vector<int64_t> ev;
        const int r = device_select2d_lag(ds, {method}, {Gm}, {th0}, max_iter, tho, fo, ev);
        if (r != KDEFFT_OK) return r;
        th_out = tho[0];
        f_out = fo[0];
        *evals_out = ev[0];
        return KDEFFT_OK;
    }
    auto pmin = [](int m) { return (int)next_smooth(m); };
    // cluster size, batch size and support cap from the shared-memory budget
    // The two packed pairs are transformed together: the gather holds both
    // and a batch holds `chunk` lines of each.  For a cluster size and a
    // shared-memory budget, the largest support cap that fits comes first,
    // then the largest batch at that cap.
    struct Layout {
        int cs = 0, Lcap = 0, chunk = 0, gat = 0, spc = 0, cap = 0, pmax = 0;
    };
    auto size_for = [&](int cs, size_t budget, Layout& lay) {
        int Lcap = std::max(M0, M1) - 1;
        for (;;) {
            const int L0 = std::min(Lcap, M0 - 1), L1 = std::min(Lcap, M1 - 1);
            const int P0 = pmin(M0 + L0), P1 = pmin(M1 + L1);
            if (P0 <= MAXP && P1 <= MAXP) {
                const int cpc = (P1 / 2 + 1 + cs - 1) / cs;
                const int gat = (2 * (2 * std::max(L0, L1) + 1) * cpc + 1) & ~1;
                const int spc = cpc * P0, pmax = std::max(P0, P1);
                for (int chunk = 8; chunk >= 3; --chunk) {
                    const int cap = 2 * chunk * pmax;
                    const size_t need =
                        sizeof(float2) * (size_t)(gat + 2 * pmax + 2 * (cap + cap / 16 + 1)) + sizeof(float) * spc;
                    if (need <= budget) {
                        lay = Layout{cs, Lcap, chunk, gat, spc, cap, pmax};
                        return true;
                    }
                }
            }
            if (Lcap <= 8) return false;
            Lcap = Lcap * 3 / 4;
        }
    };
    // 16-CTA clusters, two CTAs per SM.  (Measured: smaller clusters, which
    // let every start of a 16-start search be resident at once, lose more to
    // the larger share of each CTA than they gain from the absent second
    // wave.)
    Layout lay;
    if (!size_for(16, 110 * 1024, lay)) return KDEFFT_ERR_UNSUPPORTED;
    const int cs = lay.cs, Lcap = lay.Lcap, chunk = lay.chunk, gat = lay.gat, spc = lay.spc, cap = lay.cap,
              pmax = lay.pmax;
    // the (L0, L1) pairs met as lambda grows: breakpoints of ceil(tau s / delta_k)
    std::vector<double> brk;
    for (int k = 0; k < 2; ++k)
        for (int m = 0; m <= Lcap + 1; ++m) brk.push_back(m * ds->delta[k] / ds->opts.tau);
    std::sort(brk.begin(), brk.end());
    std::vector<std::array<int, 4>> pairsP;
    std::set<std::pair<int, int>> seenP;
    auto Lof = [&](double sq, int k) {
        double v = std::ceil(ds->opts.tau * sq / ds->delta[k]);
        const double cap_ = (double)(ds->M[k] - 1);
        if (!(v <= cap_)) v = cap_;
        if (v < 1.0) v = 1.0;
        return (int)v;
    };
    for (size_t i = 0; i + 1 < brk.size(); ++i)
        for (double t : {0.0, 0.5, 1.0}) {
            const double sq = brk[i] + t * (brk[i + 1] - brk[i]);
            const int L0 = Lof(sq, 0), L1 = Lof(sq, 1);
            if (L0 > Lcap || L1 > Lcap) continue;
            const int P0 = pmin(M0 + L0), P1 = pmin(M1 + L1);
            if (seenP.insert({P0, P1}).second) pairsP.push_back({P0, P1, 0, 0});
        }
    if (pairsP.empty() || pairsP.size() > 256) return KDEFFT_ERR_UNSUPPORTED;
    {
        std::vector<std::pair<kdefft_ds, std::array<int, 4>>> need;
        for (auto& pp : pairsP) need.push_back({ds, pp});
        KCHK(ensure_spectra<float>(c, need));
    }
    std::vector<SelSpec> specs;
    for (auto& pp : pairsP) {
        SelSpec sp{};
        sp.P0 = pp[0];
        sp.P1 = pp[1];
        if (!radix_plan(sp.P0, sp.a0, 32) || !radix_plan(sp.P1, sp.a1, 32)) return KDEFFT_ERR_UNSUPPORTED;
        sp.a0.tw_off = twiddle_offset(c, sp.P0);
        sp.a1.tw_off = twiddle_offset(c, sp.P1);
        auto it = ds->spectra.find(spectrum_key(ds, pp.data(), sizeof(float)));
        if (it == ds->spectra.end()) return fail(KDEFFT_ERR_CUDA, "count spectrum missing");
        sp.spec = (const float*)it->second->p;
        sp.scale = 1.0 / ((double)ds->n * (double)ds->n * (double)sp.P0 * (double)sp.P1);
        {   // two packed pairs: S_0 axis-1 lines and Q_1 axis-0 columns each, one read of the spectrum
            const double P0d = sp.P0, P1d = sp.P1, Q1 = std::floor(P1d / 2) + 1;
            sp.fl_line = 2.0 * 5.0 * P1d * std::log2(P1d);
            sp.fl_fix = 2.0 * Q1 * (5.0 * P0d * std::log2(P0d) + 4.0 * P0d);
            sp.by = Q1 * P0d * sizeof(float);
        }
        specs.push_back(sp);
    }
    KCHK(sync_twiddles(c));
    std::vector<int> ptab(2 * (Lcap + 1));
    for (int L = 0; L <= Lcap; ++L) {
        ptab[L] = pmin(M0 + L);
        ptab[Lcap + 1 + L] = pmin(M1 + L);
    }
    // device tables: specs | ptab | starts
    const size_t bS = sizeof(SelSpec) * specs.size(), bP = sizeof(int) * ptab.size(), bT = sizeof(SelStart) * nst;
    const size_t oP = (bS + 255) & ~(size_t)255, oT = (oP + bP + 255) & ~(size_t)255;
    KCHK(c->sel_buf.ensure(oT + bT));
    std::vector<unsigned char> hb(oT + bT, 0);
    std::memcpy(hb.data(), specs.data(), bS);
    std::memcpy(hb.data() + oP, ptab.data(), bP);
    std::vector<SelStart> st(nst);
    for (int i = 0; i < nst; ++i) {
        std::memset(&st[i], 0, sizeof(SelStart));
        for (int k = 0; k < 3; ++k) st[i].th[k] = th0[i][k];
    }
    std::memcpy(hb.data() + oT, st.data(), bT);
    unsigned char* db = (unsigned char*)c->sel_buf.p;
    KCU(cudaMemcpyAsync(db, hb.data(), hb.size(), cudaMemcpyHostToDevice, c->stream));
    c->h2d += (int64_t)hb.size();
    SelectParams prm{};
    prm.method = (method == KDEFFT_LSCV) ? 0 : 1;
    prm.max_iter = max_iter;
    prm.cs = cs;
    prm.nspec = (int)specs.size();
    prm.widest = (method == KDEFFT_LSCV && ds->opts.L_basis == KDEFFT_L_WIDEST) ? 1 : 0;
    prm.M0 = M0;
    prm.M1 = M1;
    prm.Lcap = Lcap;
    prm.Lcap1 = Lcap;
    prm.chunk = chunk;
    prm.gat_elems = gat;
    prm.spc_elems = (spc + 3) & ~3;
    prm.cap = cap;
    prm.pmax = pmax;
    prm.n = (double)ds->n;
    prm.inv_n = 1.0 / prm.n;
    prm.inv_n2 = 1.0 / (prm.n * prm.n);
    prm.inv_nf = (float)prm.inv_n;
    prm.inv_n2h = (float)prm.inv_n2;
    prm.inv_n2l = (float)(prm.inv_n2 - (double)prm.inv_n2h);
    prm.tau = ds->opts.tau;
    prm.delta0 = ds->delta[0];
    prm.delta1 = ds->delta[1];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) prm.G[a * 2 + b] = (method == KDEFFT_SCV) ? Gm(a, b) : 0.0;
    params_f32(prm);
    prm.ptab0 = (const int*)(db + oP);
    prm.ptab1 = (const int*)(db + oP) + (Lcap + 1);
    prm.specs = (const SelSpec*)db;
    prm.errflag = c->errflag;
    prm.rec = c->rec;
    prm.rec_cap = c->rec_cap;
    if (c->rec && (int64_t)nst * c->rec_cap * SEL_REC > c->rec_len)
        return fail(KDEFFT_ERR_ARG, "search record buffer smaller than starts x cap x fields");
    cudaEvent_t ev = prof_start(c);
    cudaError_t le = launch_select2d(prm, (SelStart*)(db + oT), nst, (const float2*)c->tw32.p, c->stream);
    if (le == cudaErrorNotSupported) return KDEFFT_ERR_UNSUPPORTED;
    KCU(le);
    prof_stop(c, ev, "select2d_f32", 0.0, 0.0);
    KCU(cudaMemcpyAsync(st.data(), db + oT, bT, cudaMemcpyDeviceToHost, c->stream));
    {
        HostTimer w(c, "host:wait");
        KCU(cudaStreamSynchronize(c->stream));
    }
    c->d2h += (int64_t)bT;
    if (c->prof && !c->pending.empty() && ev) {   // the work is known once the searches have ended
        double fl = 0.0, by = 0.0;
        for (const SelStart& s : st) {
            fl += s.flops;
            by += s.bytes;
        }
        c->pending.back().flops = fl;
        c->pending.back().bytes = by;
    }
    prof_flush(c);
    KCHK(check_errflag(c));
    th_out.assign(nst, std::vector<double>(3));
    f_out.assign(nst, INFINITY);
    int64_t ev_total = 0;
    for (int i = 0; i < nst; ++i) {
        for (int k = 0; k < 3; ++k) th_out[i][k] = st[i].th[k];
        f_out[i] = st[i].f;
        ev_total += st[i].evals;
    }
    *evals_out = ev_total;
    return KDEFFT_OK;
}

// Backtracking, as in the device-resident search: a rejected trial step is
// replaced by the minimiser of the quadratic through f(0), the slope and
// f(step), kept within [0.1, 0.5] of the step (a point outside the domain
// halves it).  The line search gives up after kMaxBacktracks rejections, or
// once the next trial point would move theta by less than kStepFloor in every
// coordinate (about 2e-5 relative in H), which the FP32 objective cannot
// resolve: the binned objective steps where a support L_k changes with H
// (Eq. 26), and a sufficient-decrease test at smaller steps only measures
// those steps.
static constexpr int kMaxBacktracks = 12;
static constexpr double kStepFloor = 1e-5;

// Start points of the multi-start search: Hstart, then dilations (factors
// 2^{-1}..2^{1} in half powers of two) and plane rotations of it.
static std::vector<Mat> start_bandwidths(const Mat& Hstart, int n_starts) {
    const int d = Hstart.d;
    std::vector<Mat> out(n_starts, Hstart);
    for (int s = 1; s < n_starts; ++s) {
        const double fac = std::pow(2.0, ((s % 5) - 2) * 0.5);
        const double ang = 0.35 * s;
        const int a = (s - 1) % std::max(1, d - 1), b = (d > 1) ? a + 1 : a;
        Mat Rt;
        Rt.d = d;
        for (int i = 0; i < d; ++i) Rt(i, i) = 1.0;
        if (d > 1) {
            Rt(a, a) = std::cos(ang);
            Rt(b, b) = std::cos(ang);
            Rt(a, b) = -std::sin(ang);
            Rt(b, a) = std::sin(ang);
        }
        Mat T;
        T.d = d;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                double sum = 0.0;
                for (int k = 0; k < d; ++k)
                    for (int l = 0; l < d; ++l) sum += Rt(i, k) * Hstart(k, l) * Rt(j, l);
                T(i, j) = fac * sum;
            }
        out[s] = T;
    }
    return out;
}

// End of a device-resident search: the best start's end point, and the
// objective there through the regular evaluation path (the search compared
// its own FP32 values; SCV takes the FP64 route for its cancelling terms).
// The LSCV value is evaluated with its gradient, as a caller checking
// stationarity asks for it.
static int device_best(kdefft_ds ds, const std::vector<std::vector<double>>& tho, const std::vector<double>& fo,
                       double* H_out) {
    const int d = ds->d;
    const Opt o{d, class_params(d, KDEFFT_H_FULL)};
    int best = 0;
    for (int s = 1; s < (int)fo.size(); ++s)
        if (fo[s] < fo[best]) best = s;
    if (!std::isfinite(fo[best])) return fail(KDEFFT_ERR_ARG, "no start point inside the search domain");
    Mat Hb = theta_to_H(o, tho[best].data());
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) H_out[a * d + b] = Hb(a, b);
    return KDEFFT_OK;
}

static int finish_device_select(kdefft_ds ds, int method, const Mat& Gm, const std::vector<std::vector<double>>& tho,
                                const std::vector<double>& fo, int64_t dev_evals, double* H_out, double* f_out,
                                int64_t* n_evals) {
    KCHK(device_best(ds, tho, fo, H_out));
    std::vector<double> v, gdummy;
    if (method == KDEFFT_SCV)
        KCHK(eval_scv(ds, H_out, 1, Gm, v, nullptr, /*split64=*/true));
    else
        KCHK(eval_lscv(ds, H_out, 1, v, &gdummy));
    if (f_out) *f_out = v[0];
    if (n_evals) *n_evals = dev_evals + 1;
    return KDEFFT_OK;
}

static int select_H_impl(kdefft_ds ds, int method, const double* H0, const double* G, int n_starts, int max_iter,
                         bool nelder_mead, double* H_out, double* f_out, int64_t* n_evals, int hclass = KDEFFT_H_FULL) {
    if (!ds || !H_out) return fail(KDEFFT_ERR_ARG, "NULL argument");
    if (method != KDEFFT_LSCV && method != KDEFFT_SCV && method != KDEFFT_PI)
        return fail(KDEFFT_ERR_ARG, "unknown method");
    if (n_starts < 1) n_starts = 1;
    if (max_iter < 1) max_iter = nelder_mead ? 500 : 100;
    KCU(cudaSetDevice(ds->ctx->device));
    const int d = ds->d;
    if (hclass != KDEFFT_H_FULL && hclass != KDEFFT_H_DIAG && hclass != KDEFFT_H_SCALAR)
        return fail(KDEFFT_ERR_ARG, "unknown bandwidth class");
    Opt o{d, class_params(d, hclass), hclass};
    const int p = o.p;
    Mat Hstart;
    if (H0) {
        KCHK(sym_check(H0, d, Hstart, "H0"));
    } else {
        KCHK(get_G(ds, nullptr, Hstart));
    }
    KCHK(spd_or_fail(Hstart, "H0"));
    Mat Gm;
    if (method != KDEFFT_LSCV) KCHK(get_G(ds, G, Gm));
    std::vector<double> psi4;
    if (method == KDEFFT_PI) KCHK(psi4_kron(ds, Gm, psi4));
    int64_t evals = 0;

    // Domain of the search: H numerically SPD and resolvable by the grid,
    // sqrt(H_kk) >= delta_k / 2 on every axis.  With binned data the objective
    // is unbounded below as H -> 0 (a bin holding several points contributes
    // a diagonal term of order -phi_H(0)), so bandwidths finer than the bins
    // are outside the domain: such a trial point counts as f = +inf.
    auto in_domain = [&](const Mat& H) {
        Mat Lc;
        if (!cholesky(H, Lc)) return false;
        for (int k = 0; k < d; ++k)
            if (!(std::sqrt(H(k, k)) >= 0.5 * ds->delta[k]) || !std::isfinite(H(k, k))) return false;
        return true;
    };
    // batched evaluation of value + theta-gradient for a list of theta
    auto evaluate = [&](const std::vector<std::vector<double>>& ths, std::vector<double>& f,
                        std::vector<std::vector<double>>& gt) -> int {
        HostTimer ht(ds->ctx, "host:eval");
        const int m = (int)ths.size();
        f.assign(m, INFINITY);
        gt.assign(m, std::vector<double>(p, 0.0));
        std::vector<int> idx;
        std::vector<double> Hs;
        for (int i = 0; i < m; ++i) {
            Mat H = theta_to_H(o, ths[i].data());
            if (!in_domain(H)) continue;
            idx.push_back(i);
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) Hs.push_back(H(a, b));
        }
        const int mv = (int)idx.size();
        if (mv == 0) return KDEFFT_OK;
        std::vector<double> v, g;
        int r;
        if (method == KDEFFT_LSCV)
            r = eval_lscv(ds, Hs.data(), mv, v, &g);
        else if (method == KDEFFT_SCV)
            r = eval_scv(ds, Hs.data(), mv, Gm, v, &g, /*split64=*/false);
        else
            r = eval_pi(ds, Hs.data(), mv, psi4, v, &g);
        if (r != KDEFFT_OK) return r;
        evals += mv;
        for (int j = 0; j < mv; ++j) {
            const int i = idx[j];
            f[i] = v[j];
            grad_theta(o, ths[i].data(), g.data() + (size_t)j * d * d, gt[i].data());
        }
        return KDEFFT_OK;
    };

    // batched evaluation of values only
    auto evaluate_values = [&](const std::vector<std::vector<double>>& ths, std::vector<double>& f) -> int {
        HostTimer ht(ds->ctx, "host:eval");
        const int m = (int)ths.size();
        f.assign(m, INFINITY);
        std::vector<int> idx;
        std::vector<double> Hs;
        for (int i = 0; i < m; ++i) {
            Mat H = theta_to_H(o, ths[i].data());
            if (!in_domain(H)) continue;
            idx.push_back(i);
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) Hs.push_back(H(a, b));
        }
        const int mv = (int)idx.size();
        if (mv == 0) return KDEFFT_OK;
        std::vector<double> v;
        int r;
        if (method == KDEFFT_LSCV)
            r = eval_lscv(ds, Hs.data(), mv, v, nullptr);
        else if (method == KDEFFT_SCV)
            r = eval_scv(ds, Hs.data(), mv, Gm, v, nullptr, /*split64=*/false);
        else
            r = eval_pi(ds, Hs.data(), mv, psi4, v, nullptr);
        if (r != KDEFFT_OK) return r;
        evals += mv;
        for (int j = 0; j < mv; ++j) f[idx[j]] = v[j];
        return KDEFFT_OK;
    };

    // start points: Hstart, then dilations and plane rotations of it
    struct State {
        std::vector<double> th, g, dir, Binv, th_try;
        double f = 0.0, step = 1.0, slope = 0.0;
        double dfp = 0.0;   // decrease of the last accepted step (0: none since the last reset)
        int iter = 0, ls = 0;
        bool done = false;
        bool fresh = true;   // the current direction comes from a reset (scaled steepest descent)
    };
    std::vector<State> st(n_starts);
    {
        const std::vector<Mat> Hs0 = start_bandwidths(Hstart, n_starts);
        for (int s = 0; s < n_starts; ++s) {
            st[s].th.resize(p);
            H_to_theta(o, Hs0[s], st[s].th.data());
            st[s].Binv.assign((size_t)p * p, 0.0);
            for (int i = 0; i < p; ++i) st[s].Binv[i * p + i] = 1.0;
        }
    }
    // the reported value at the chosen point: SCV iterations compare FP32
    // values, the reported one takes the FP64 route for the cancelling terms
    auto report = [&](const std::vector<double>& th, double f) -> int {
        if (!std::isfinite(f)) return fail(KDEFFT_ERR_ARG, "no start point inside the search domain");
        Mat Hb = theta_to_H(o, th.data());
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) H_out[a * d + b] = Hb(a, b);
        if (method == KDEFFT_SCV) {
            std::vector<double> v;
            KCHK(eval_scv(ds, H_out, 1, Gm, v, nullptr, /*split64=*/true));
            f = v[0];
        }
        if (f_out) *f_out = f;
        if (n_evals) *n_evals = evals;
        return KDEFFT_OK;
    };
    if (nelder_mead) {
        // Nelder-Mead on theta with the factors of Sec. 6 (reflection 1,
        // contraction 0.5, expansion 2; shrink towards the best vertex by
        // the contraction factor), initial simplex theta_0 + 0.1 e_i, stop
        // when f_worst - f_best <= reltol (|f_best| + reltol) with
        // reltol = 2^-26 or after max_iter objective evaluations per start.
        // Starts run in lock-step: every round evaluates the pending points
        // of all starts in one batched call (values only).
        const double alpha = 1.0, beta = 0.5, gamma = 2.0, reltol = 1.4901161193847656e-8;
        struct NM {
            std::vector<std::vector<double>> x, pend;
            std::vector<double> fx, c, xr, xe, xc;
            double fr = 0.0;
            int phase = 0, nev = 0, worst = 0, second = 0, best = 0;
            bool outside = false, done = false;
        };
        std::vector<NM> nm(n_starts);
        for (int s = 0; s < n_starts; ++s) {
            NM& q = nm[s];
            q.x.assign(p + 1, st[s].th);
            for (int i = 0; i < p; ++i) q.x[i + 1][i] += 0.1;
            q.pend = q.x;
            q.fx.assign(p + 1, INFINITY);
        }
        auto lin = [&](const std::vector<double>& a, const std::vector<double>& b, double t) {
            std::vector<double> r(p);
            for (int i = 0; i < p; ++i) r[i] = a[i] + t * (b[i] - a[i]);   // a + t (b - a)
            return r;
        };
        auto begin_iteration = [&](NM& q) {
            q.best = q.worst = 0;
            for (int i = 1; i <= p; ++i) {
                if (q.fx[i] < q.fx[q.best]) q.best = i;
                if (q.fx[i] >= q.fx[q.worst]) q.worst = i;
            }
            q.second = (q.worst == q.best) ? (q.best + 1) % (p + 1) : q.best;
            for (int i = 0; i <= p; ++i)
                if (i != q.worst && q.fx[i] >= q.fx[q.second]) q.second = i;
            const double fb = q.fx[q.best], fw = q.fx[q.worst];
            if (!std::isfinite(fb) || q.nev >= max_iter || (std::isfinite(fw) && fw - fb <= reltol * (std::fabs(fb) + reltol))) {
                q.done = true;
                q.pend.clear();
                return;
            }
            q.c.assign(p, 0.0);
            for (int i = 0; i <= p; ++i)
                if (i != q.worst)
                    for (int k = 0; k < p; ++k) q.c[k] += q.x[i][k] / p;
            q.xr = lin(q.c, q.x[q.worst], -alpha);   // c + alpha (c - x_worst)
            q.pend = {q.xr};
            q.phase = 1;
        };
        auto consume = [&](NM& q, const std::vector<double>& v) {
            q.nev += (int)v.size();
            switch (q.phase) {
                case 0:
                    q.fx = v;
                    begin_iteration(q);
                    break;
                case 1:
                    q.fr = v[0];
                    if (q.fr < q.fx[q.best]) {
                        q.xe = lin(q.c, q.xr, gamma);   // c + gamma (x_r - c)
                        q.pend = {q.xe};
                        q.phase = 2;
                    } else if (q.fr < q.fx[q.second]) {
                        q.x[q.worst] = q.xr;
                        q.fx[q.worst] = q.fr;
                        begin_iteration(q);
                    } else {
                        q.outside = q.fr < q.fx[q.worst];
                        q.xc = q.outside ? lin(q.c, q.xr, beta) : lin(q.c, q.x[q.worst], beta);
                        q.pend = {q.xc};
                        q.phase = 3;
                    }
                    break;
                case 2:
                    if (v[0] < q.fr) {
                        q.x[q.worst] = q.xe;
                        q.fx[q.worst] = v[0];
                    } else {
                        q.x[q.worst] = q.xr;
                        q.fx[q.worst] = q.fr;
                    }
                    begin_iteration(q);
                    break;
                case 3:
                    if (q.outside ? v[0] <= q.fr : v[0] < q.fx[q.worst]) {
                        q.x[q.worst] = q.xc;
                        q.fx[q.worst] = v[0];
                        begin_iteration(q);
                    } else {
                        q.pend.clear();
                        for (int i = 0; i <= p; ++i)
                            if (i != q.best) {
                                q.x[i] = lin(q.x[q.best], q.x[i], beta);
                                q.pend.push_back(q.x[i]);
                            }
                        q.phase = 4;
                    }
                    break;
                default: {
                    int k = 0;
                    for (int i = 0; i <= p; ++i)
                        if (i != q.best) q.fx[i] = v[k++];
                    begin_iteration(q);
                }
            }
        };
        for (int round = 0; round < 4 * max_iter + 8; ++round) {
            std::vector<std::vector<double>> ths;
            std::vector<std::pair<int, int>> owner;   // (start, count)
            for (int s = 0; s < n_starts; ++s)
                if (!nm[s].done && !nm[s].pend.empty()) {
                    owner.push_back({s, (int)nm[s].pend.size()});
                    for (auto& t : nm[s].pend) ths.push_back(t);
                }
            if (owner.empty()) break;
            std::vector<double> f;
            KCHK(evaluate_values(ths, f));
            size_t k = 0;
            for (auto& ow : owner) {
                std::vector<double> v(f.begin() + k, f.begin() + k + ow.second);
                k += ow.second;
                consume(nm[ow.first], v);
            }
        }
        int bs = 0, bv = 0;
        double fb = INFINITY;
        for (int s = 0; s < n_starts; ++s)
            for (int i = 0; i <= p; ++i)
                if (nm[s].fx[i] < fb) {
                    fb = nm[s].fx[i];
                    bs = s;
                    bv = i;
                }
        return report(nm[bs].x[bv], fb);
    }
    if (d == 2 && hclass == KDEFFT_H_FULL) {
        std::vector<std::vector<double>> ths, tho;
        for (auto& s : st) ths.push_back(s.th);
        std::vector<double> fo;
        int64_t dev_evals = 0;
        const int r = device_select2d(ds, method, Gm, ths, max_iter, tho, fo, &dev_evals);
        if (r == KDEFFT_OK) return finish_device_select(ds, method, Gm, tho, fo, dev_evals, H_out, f_out, n_evals);
        if (r != KDEFFT_ERR_UNSUPPORTED) return r;
    }
    {
        std::vector<std::vector<double>> ths;
        for (auto& s : st) ths.push_back(s.th);
        std::vector<double> f;
        std::vector<std::vector<double>> g;
        KCHK(evaluate(ths, f, g));
        for (int s = 0; s < n_starts; ++s) {
            st[s].f = f[s];
            st[s].g = g[s];
            if (!std::isfinite(f[s])) st[s].done = true;
            // initial inverse-Hessian scale: a unit step moves theta by ~0.1
            double gn = 0.0;
            for (double v : g[s]) gn = std::max(gn, std::fabs(v));
            const double sc = (gn > 0) ? 0.1 / gn : 1.0;
            for (int i = 0; i < p; ++i) st[s].Binv[i * p + i] = sc;
        }
    }
    auto new_direction = [&](State& s) {
        s.dir.assign(p, 0.0);
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) s.dir[i] -= s.Binv[i * p + j] * s.g[j];
        s.slope = 0.0;
        for (int i = 0; i < p; ++i) s.slope += s.dir[i] * s.g[i];
        if (!(s.slope < 0.0)) {   // not a descent direction: reset to steepest descent
            double gn = 0.0;
            for (double v : s.g) gn = std::max(gn, std::fabs(v));
            const double sc = (gn > 0) ? 0.1 / gn : 1.0;
            std::fill(s.Binv.begin(), s.Binv.end(), 0.0);
            for (int i = 0; i < p; ++i) {
                s.Binv[i * p + i] = sc;
                s.dir[i] = -sc * s.g[i];
            }
            s.slope = 0.0;
            for (int i = 0; i < p; ++i) s.slope += s.dir[i] * s.g[i];
        }
        double dm = 0.0;
        for (double v : s.dir) dm = std::max(dm, std::fabs(v));
        if (dm > 1.0) {   // at most a factor e per iteration on the Cholesky diagonal
            for (double& v : s.dir) v /= dm;
            s.slope /= dm;
        }
        // first trial step: the minimiser of the quadratic that repeats the
        // last accepted decrease along the new direction (Nocedal & Wright),
        // 1.01 x 2 (f_k - f_{k-1}) / slope, at most the unit quasi-Newton step
        s.step = 1.0;
        if (s.dfp < 0.0) {
            const double q = 2.02 * s.dfp / s.slope;
            if (q > 0.0) s.step = std::min(1.0, q);
        }
        s.ls = 0;
        s.th_try.resize(p);
        for (int i = 0; i < p; ++i) s.th_try[i] = s.th[i] + s.step * s.dir[i];
    };
    for (auto& s : st) {
        if (s.done) continue;
        double gn = 0.0;
        for (double v : s.g) gn = std::max(gn, std::fabs(v));
        if (gn == 0.0) s.done = true;
        else new_direction(s);
    }
    for (int round = 0; round < 40 * max_iter; ++round) {
        std::vector<int> act;
        std::vector<std::vector<double>> ths;
        for (int s = 0; s < n_starts; ++s)
            if (!st[s].done) {
                act.push_back(s);
                ths.push_back(st[s].th_try);
            }
        if (act.empty()) break;
        std::vector<double> f;
        std::vector<std::vector<double>> g;
        KCHK(evaluate(ths, f, g));
        for (size_t k = 0; k < act.size(); ++k) {
            State& s = st[act[k]];
            const double fn = f[k];
            if (std::isfinite(fn) && fn <= s.f + 1e-4 * s.step * s.slope) {
                // accept: BFGS update of the inverse Hessian
                std::vector<double> sv(p), yv(p);
                for (int i = 0; i < p; ++i) {
                    sv[i] = s.th_try[i] - s.th[i];
                    yv[i] = g[k][i] - s.g[i];
                }
                double sy = 0.0;
                for (int i = 0; i < p; ++i) sy += sv[i] * yv[i];
                if (sy > 1e-300) {
                    std::vector<double> By(p, 0.0);
                    for (int i = 0; i < p; ++i)
                        for (int j = 0; j < p; ++j) By[i] += s.Binv[i * p + j] * yv[j];
                    double yBy = 0.0;
                    for (int i = 0; i < p; ++i) yBy += yv[i] * By[i];
                    for (int i = 0; i < p; ++i)
                        for (int j = 0; j < p; ++j)
                            s.Binv[i * p + j] += ((sy + yBy) * sv[i] * sv[j]) / (sy * sy) -
                                                 (By[i] * sv[j] + sv[i] * By[j]) / sy;
                }
                const double fold = s.f;
                s.th = s.th_try;
                s.f = fn;
                s.dfp = fn - fold;
                s.g = g[k];
                s.iter++;
                double gn = 0.0, tn = 0.0;
                for (int i = 0; i < p; ++i) {
                    gn = std::max(gn, std::fabs(s.g[i]));
                    tn = std::max(tn, std::fabs(sv[i]));
                }
                if (s.iter >= max_iter || std::fabs(fold - fn) <= 1e-12 * std::fabs(fn) + 1e-300 || tn < 1e-10 ||
                    gn < 1e-12 * (std::fabs(fn) + 1e-300)) {
                    s.done = true;
                } else {
                    s.fresh = false;
                    new_direction(s);
                }
            } else {
                double nstep = 0.5 * s.step;
                if (std::isfinite(fn)) {
                    const double pred = s.step * s.slope, den = (fn - s.f) - pred;
                    if (den > 0.0) nstep = std::min(std::max(-0.5 * pred * s.step / den, 0.1 * s.step), 0.5 * s.step);
                }
                s.step = nstep;
                s.ls++;
                double dm = 0.0;
                for (double v : s.dir) dm = std::max(dm, std::fabs(v));
                const bool give_up = s.ls > kMaxBacktracks || s.step * dm < kStepFloor;
                if (give_up && !s.fresh) {
                    // restart: the quasi-Newton model failed here; scaled steepest descent once
                    double gm = 0.0;
                    for (double v : s.g) gm = std::max(gm, std::fabs(v));
                    const double sc = (gm > 0) ? 0.1 / gm : 1.0;
                    std::fill(s.Binv.begin(), s.Binv.end(), 0.0);
                    for (int i = 0; i < p; ++i) s.Binv[i * p + i] = sc;
                    s.fresh = true;
                    s.dfp = 0.0;
                    new_direction(s);
                } else if (give_up) {
                    s.done = true;
                } else {
                    for (int i = 0; i < p; ++i) s.th_try[i] = s.th[i] + s.step * s.dir[i];
                }
            }
        }
    }
    int best = 0;
    for (int s = 1; s < n_starts; ++s)
        if (st[s].f < st[best].f) best = s;
    return report(st[best].th, st[best].f);
}

extern "C" int kdefft_select_H(kdefft_ds ds, int method, const double* H0, const double* G, int n_starts,
                               int max_iter, double* H_out, double* f_out, int64_t* n_evals) {
    return select_H_impl(ds, method, H0, G, n_starts, max_iter, false, H_out, f_out, n_evals);
}

extern "C" int kdefft_select_H_multi(kdefft_ds ds, int nmethods, const int* methods, const double* H0,
                                     const double* G, int n_starts, int max_iter, double* H_out, double* f_out,
                                     int64_t* n_evals) {
    if (!ds || !methods || !H_out || nmethods < 1) return fail(KDEFFT_ERR_ARG, "NULL argument or no criterion");
    for (int m = 0; m < nmethods; ++m)
        if (methods[m] != KDEFFT_LSCV && methods[m] != KDEFFT_SCV && methods[m] != KDEFFT_PI)
            return fail(KDEFFT_ERR_ARG, "unknown method");
    KCU(cudaSetDevice(ds->ctx->device));
    const int d = ds->d;
    if (n_starts < 1) n_starts = 1;
    if (max_iter < 1) max_iter = 100;
    // criteria the device-resident search covers go pairwise into one launch;
    // the others run one after another
    std::vector<int> dev, host;
    for (int m = 0; m < nmethods; ++m)
        (ds->ctx->lag && select2d_covered(ds, methods[m]) ? dev : host).push_back(m);
    if (!dev.empty()) {
        Mat Hstart;
        if (H0) {
            KCHK(sym_check(H0, d, Hstart, "H0"));
        } else {
            KCHK(get_G(ds, nullptr, Hstart));
        }
        KCHK(spd_or_fail(Hstart, "H0"));
        const Opt o{d, class_params(d, KDEFFT_H_FULL)};
        std::vector<std::vector<double>> th0;
        for (const Mat& H : start_bandwidths(Hstart, n_starts)) {
            std::vector<double> th(o.p);
            H_to_theta(o, H, th.data());
            th0.push_back(th);
        }
        for (size_t k = 0; k < dev.size(); k += 2) {
            std::vector<int> ms, idx;
            std::vector<Mat> Gms;
            for (size_t q = k; q < std::min(dev.size(), k + 2); ++q) {
                const int m = dev[q];
                Mat Gm;
                if (methods[m] != KDEFFT_LSCV) KCHK(get_G(ds, G, Gm));
                ms.push_back(methods[m]);
                idx.push_back(m);
                Gms.push_back(Gm);
            }
            std::vector<std::vector<std::vector<double>>> tho;
            std::vector<std::vector<double>> fo;
            std::vector<int64_t> ev;
            const int r = device_select2d_lag(ds, ms, Gms, std::vector<std::vector<std::vector<double>>>(ms.size(), th0),
                                              max_iter, tho, fo, ev);
            if (r == KDEFFT_ERR_UNSUPPORTED) {
                for (int m : idx) host.push_back(m);
                continue;
            }
            KCHK(r);
            if (ms.size() == 2 && ms[0] != ms[1]) {
                // LSCV and SCV: both end-point values (the same requests as
                // finish_device_select's) in one run, one wait
                const int qL = ms[0] == KDEFFT_LSCV ? 0 : 1, qS = 1 - qL;
                double* HL = H_out + (size_t)idx[qL] * d * d;
                double* HS = H_out + (size_t)idx[qS] * d * d;
                KCHK(device_best(ds, tho[qL], fo[qL], HL));
                KCHK(device_best(ds, tho[qS], fo[qS], HS));
                ReqSet rs;
                LscvJob jl;
                ScvJob js;
                KCHK(lscv_requests(rs, ds, HL, 1, true, jl));
                KCHK(scv_requests(rs, ds, HS, 1, Gms[qS], false, /*split64=*/true, js));
                KCHK(run(ds->ctx, rs));
                std::vector<double> vl, gl, vs;
                lscv_assemble(rs, ds, jl, vl, &gl);
                scv_assemble(rs, ds, js, vs, nullptr);
                if (f_out) {
                    f_out[idx[qL]] = vl[0];
                    f_out[idx[qS]] = vs[0];
                }
                if (n_evals) {
                    n_evals[idx[qL]] = ev[qL] + 1;
                    n_evals[idx[qS]] = ev[qS] + 1;
                }
            } else {
                for (size_t q = 0; q < ms.size(); ++q) {
                    const int m = idx[q];
                    KCHK(finish_device_select(ds, ms[q], Gms[q], tho[q], fo[q], ev[q], H_out + (size_t)m * d * d,
                                              f_out ? f_out + m : nullptr, n_evals ? n_evals + m : nullptr));
                }
            }
        }
    }
    for (int m : host)
        KCHK(select_H_impl(ds, methods[m], H0, G, n_starts, max_iter, false, H_out + (size_t)m * d * d,
                           f_out ? f_out + m : nullptr, n_evals ? n_evals + m : nullptr));
    return KDEFFT_OK;
}

extern "C" int kdefft_select_H_nm(kdefft_ds ds, int method, const double* H0, const double* G, int n_starts,
                                  int max_iter, double* H_out, double* f_out, int64_t* n_evals) {
    return select_H_impl(ds, method, H0, G, n_starts, max_iter, true, H_out, f_out, n_evals);
}

extern "C" int kdefft_select_H_class(kdefft_ds ds, int method, int hclass, int optimizer, const double* H0,
                                     const double* G, int n_starts, int max_iter, double* H_out, double* f_out,
                                     int64_t* n_evals) {
    if (optimizer != 0 && optimizer != 1) return fail(KDEFFT_ERR_ARG, "optimizer: 0 quasi-Newton, 1 Nelder-Mead");
    return select_H_impl(ds, method, H0, G, n_starts, max_iter, optimizer == 1, H_out, f_out, n_evals, hclass);
}
