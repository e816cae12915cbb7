// libsht C ABI: plans (ring geometry, recurrence tables, twiddle tables) and
// the alm2map / map2alm_adjoint entry points declared in include/sht.h.
#include "sht.h"
#include "sht_internal.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <algorithm>
#include <map>
#include <queue>
#include <mutex>
#include <string>
#include <vector>

using sht::DevPlan;

struct ProfEvent {
    int stage;
    cudaEvent_t a, b;
};

struct sht_plan_s {
    int device = 0;
    bool profiling = false;
    std::vector<ProfEvent> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[SHT_NSTAGES] = {0};
    long long prof_n[SHT_NSTAGES] = {0};
    int kind = 0, lmax = 0, mmax = 0, nrings = 0, npairs = 0;
    long long nalm = 0, npix = 0;
    DevPlan dp{};
    std::vector<void *> allocs;
    void *ws = nullptr;  // Delta workspace
    size_t ws_bytes = 0;
    std::vector<int> rings_smooth_h, rings_blue_h;  // host copies of the ring lists
    std::vector<int> nphi_h;                       // pixels per ring (host copy)
    double min_sin = 0.0;                          // smallest sin(theta) over the rings
    // FP32 ring step: the register-FFT kernel's ring list and the rings left to
    // the shared-memory kernel, per kernel choice (sht_debug_ring_kernel)
    struct RfSet {
        const int *rings = nullptr, *rest_s = nullptr, *rest_b = nullptr;
        std::vector<int> rings_h, rest_s_h, rest_b_h;
    } rf_set[3];
    int rf_mode = 0;
    std::vector<int> rf_len_h;
    sht::TcWork tc;      // tensor-core forms: segment tables, status word, B-operand buffer
    size_t tc_bytes = 0;
    // tile shapes (sht_autotune): results do not depend on them
    int ring_g[2] = {2, 1};  // maps per CTA of the FP32 ring step: smooth, Bluestein ring lists
    int ring_nt = 256;       // threads per CTA of the FP32 ring step
    int fp64_bc = 8;         // maps per CTA of the FP64 Legendre step
    int fp64_ring_g = 8;     // maps per CTA of the FP64 ring step
    int adj_ring_g = 8;      // maps per CTA of the FP32 ring analysis (tensor-core transpose)
    void *lcache[4] = {};  // plan-time Lambda operand per tensor-core form (sht_lambda_cache)
    bool skip_evanescent = true;  // tensor-core forms: start items after their all-zero degrees
    void *warm = nullptr;         // the skip tables (one allocation), built on first use
    int *sched = nullptr;         // the tensor-core work lists (DevPlan::sched_off, sched_items)
    int sched_skip = -1;          // skip setting the lists were built for (-1: none yet)
    bool sched_off = false;       // test hook: round robin instead of the lists
    std::vector<int> blim_h;      // per ring block: 1 + largest order with a nonzero Delta (skip tables)
    std::vector<int> ring_mlim_h;   // per ring: the same (host copy of DevPlan::ring_mlim)
    std::vector<int2> pair_ring_h;  // (northern ring, southern ring or -1) per pair (host copy)
    std::vector<double> wring_h;  // pixel quadrature weight per ring (host copy)
    double *wring_d = nullptr;    // the same on the device (DevPlan::wring)
    // host-buffer pipeline (sht_alm2map_host): two device buffer sets, two copy
    // streams and the events that order them (created on first use)
    void *hp_buf = nullptr;
    size_t hp_bytes = 0;
    cudaStream_t hp_up = nullptr, hp_down = nullptr;
    cudaEvent_t hp_ev[8] = {};
    // index tables of the partitioned transform (sht_alm2map_mpart,
    // sht_ring_synth_part), grown on demand
    void *part_buf = nullptr;
    size_t part_bytes = 0;
    // tensor-core transpose (BF16 forms): FP32 ring analysis + operand image
    // workspace, and the (m, degree block) items, built on first use
    void *adj_ws = nullptr;
    size_t adj_bytes = 0;
    int2 *adj_items = nullptr;
    int adj_nitems = 0;
    size_t lcache_bytes[4] = {};
    std::mutex mu;
};

namespace {

thread_local std::string g_err;
std::atomic<unsigned long long> g_launches{0};

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(SHT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

constexpr int kMaxL = 8192;
constexpr int kMaxNphi = 8192;
constexpr size_t kMaxDynSmem = 227 * 1024 - 1024;  // per-CTA opt-in limit minus static use
constexpr double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------- geometry --

struct Rings {
    std::vector<double> x, s, phi0;
    std::vector<double> w;  // quadrature weight of each pixel of the ring (empty: none)
    std::vector<int> nphi, ps;
};

// Gauss-Legendre nodes by Newton iteration on P_n, northern half only and
// mirrored, so that the southern ring of each pair is exactly -x.
void gl_geometry(int n, int nphi, Rings &R)
{
    R.x.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double pa = 1.0, pb = z;  // P_{j-1}, P_j
            for (int j = 2; j <= n; ++j) {
                const double pc = ((2.0 * j - 1.0) * z * pb - (j - 1.0) * pa) / j;
                pa = pb;
                pb = pc;
            }
            const double pn = (n == 1) ? z : pb;
            const double pn1 = (n == 1) ? 1.0 : pa;
            const double dp = n * (z * pn - pn1) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        R.x[i] = z;
        R.x[n - 1 - i] = -z;
    }
    if (n % 2) R.x[n / 2] = 0.0;
    R.s.resize(n);
    for (int i = 0; i < n; ++i) R.s[i] = std::sqrt((1.0 - R.x[i]) * (1.0 + R.x[i]));
    // Gauss weight 2 / ((1 - x^2) P_n'(x)^2), times 2 pi / nphi per pixel
    R.w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        const double z = R.x[i];
        double pa = 1.0, pb = z;
        for (int j = 2; j <= n; ++j) {
            const double pc = ((2.0 * j - 1.0) * z * pb - (j - 1.0) * pa) / j;
            pa = pb;
            pb = pc;
        }
        const double pn = (n == 1) ? z : pb, pn1 = (n == 1) ? 1.0 : pa;
        const double dp = n * (z * pn - pn1) / (z * z - 1.0);
        R.w[i] = 2.0 / ((1.0 - z * z) * dp * dp) * (2.0 * kPi / nphi);
    }
    R.nphi.assign(n, nphi);
    R.phi0.assign(n, 0.0);
    R.ps.assign(n, 0);
}

// HEALPix RING geometry (Gorski et al. 2005): polar-cap ring i < nside at
// z = 1 - i^2 / (3 nside^2) with 4 i pixels starting at phi = pi / (4 i);
// equatorial ring nside <= i <= 3 nside at z = 4/3 - 2 i / (3 nside) with
// 4 nside pixels starting at phi = (pi / (4 nside)) ((i - nside + 1) mod 2).
// The southern hemisphere is the exact mirror of the northern one.
void healpix_geometry(int nside, Rings &R)
{
    const int nr = 4 * nside - 1;
    const double dn = (double)nside;
    R.x.assign(nr, 0.0);
    R.s.assign(nr, 0.0);
    R.nphi.assign(nr, 0);
    R.phi0.assign(nr, 0.0);
    R.ps.assign(nr, 0);
    for (int i = 1; i <= 2 * nside; ++i) {
        double z, s, p0;
        int np, ps;
        if (i < nside) {
            const double omz = (double)i * (double)i / (3.0 * dn * dn);
            z = 1.0 - omz;
            s = std::sqrt(omz * (2.0 - omz));
            np = 4 * i;
            ps = 1;
            p0 = kPi / (4.0 * i);
        } else {
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * dn);
            s = std::sqrt((1.0 - z) * (1.0 + z));
            np = 4 * nside;
            ps = (i - nside + 1) % 2;
            p0 = (kPi / (2.0 * dn)) * (0.5 * ps);
        }
        const int rn = i - 1, rs = nr - i;
        R.x[rn] = z;
        R.s[rn] = s;
        R.nphi[rn] = np;
        R.ps[rn] = ps;
        R.phi0[rn] = p0;
        if (rs != rn) {
            R.x[rs] = -z;
            R.s[rs] = s;
            R.nphi[rs] = np;
            R.ps[rs] = ps;
            R.phi0[rs] = p0;
        }
    }
    R.x[2 * nside - 1] = 0.0;  // equator
    R.s[2 * nside - 1] = 1.0;
    R.w.assign(nr, 4.0 * kPi / (12.0 * dn * dn));  // equal-area pixels
}

// ----------------------------------------------------------------- tables --

template <typename T>
int upload(sht_plan_s *p, const std::vector<T> &h, const T **out)
{
    *out = nullptr;
    if (h.empty()) return SHT_OK;
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, h.size() * sizeof(T));
    if (e != cudaSuccess) return fail(SHT_ENOMEM, "cudaMalloc(%zu): %s", h.size() * sizeof(T),
                                      cudaGetErrorString(e));
    p->allocs.push_back(d);
    e = cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    *out = static_cast<const T *>(d);
    return SHT_OK;
}

void free_plan(sht_plan_s *p)
{
    if (!p) return;
    {
        DeviceGuard g(p->device);
        cudaDeviceSynchronize();
        for (void *d : p->allocs) cudaFree(d);
        if (p->ws) cudaFree(p->ws);
        if (p->tc.bbuf) cudaFree(p->tc.bbuf);
        for (void *c : p->lcache)
            if (c) cudaFree(c);
        if (p->warm) cudaFree(p->warm);
        if (p->hp_buf) cudaFree(p->hp_buf);
        if (p->part_buf) cudaFree(p->part_buf);
        if (p->adj_ws) cudaFree(p->adj_ws);
        if (p->adj_items) cudaFree(p->adj_items);
        if (p->hp_up) cudaStreamDestroy(p->hp_up);
        if (p->hp_down) cudaStreamDestroy(p->hp_down);
        for (auto e : p->hp_ev)
            if (e) cudaEventDestroy(e);
        if (p->sched) cudaFree(p->sched);
        for (auto &e : p->prof_pending) {
            cudaEventDestroy(e.a);
            cudaEventDestroy(e.b);
        }
        for (auto e : p->prof_pool) cudaEventDestroy(e);
    }
    delete p;
}

// ------------------------------------------------------------ profiling --

cudaEvent_t prof_event(sht_plan_s *p)
{
    if (!p->prof_pool.empty()) {
        cudaEvent_t e = p->prof_pool.back();
        p->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one kernel launch: records events on the launch stream when the
// plan is profiling, and counts the launch.
struct StageScope {
    sht_plan_s *p;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    StageScope(sht_plan_s *p_, int stage_, cudaStream_t st_) : p(p_), stage(stage_), st(st_)
    {
        if (p->profiling) {
            a = prof_event(p);
            cudaEventRecord(a, st);
        }
    }
    void done(cudaError_t launch_rc, int kernels = 1)
    {
        if (launch_rc == cudaSuccess) g_launches.fetch_add(kernels, std::memory_order_relaxed);
        if (a) {
            cudaEvent_t b = prof_event(p);
            cudaEventRecord(b, st);
            p->prof_pending.push_back({stage, a, b});
            a = nullptr;
        }
    }
};

inline long long mofs(int lmax, int m) { return (long long)m * (2LL * lmax + 3 - m) / 2; }

int largest_prime_factor(int N)
{
    int best = 1;
    for (int p = 2; (long long)p * p <= N; ++p)
        while (N % p == 0) {
            best = p;
            N /= p;
        }
    return N > 1 ? std::max(best, N) : best;
}

// In-place iterative radix-2 FFT, forward sign, power-of-two length (plan time only).
void fft_pow2_forward(std::vector<double> &re, std::vector<double> &im)
{
    const size_t n = re.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            std::swap(re[i], re[j]);
            std::swap(im[i], im[j]);
        }
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        for (size_t k = 0; k < len / 2; ++k) {
            const double a = -2.0 * kPi * (double)k / (double)len;
            const double wr = std::cos(a), wi = std::sin(a);
            for (size_t i = k; i < n; i += len) {
                const size_t j = i + len / 2;
                const double xr = re[j] * wr - im[j] * wi;
                const double xi = re[j] * wi + im[j] * wr;
                re[j] = re[i] - xr;
                im[j] = im[i] - xi;
                re[i] += xr;
                im[i] += xi;
            }
        }
    }
}

// Point the plan's FP32 ring lists at the set of its current kernel choice.
void apply_rf_mode(sht_plan_s *p)
{
    const auto &f = p->rf_set[p->rf_mode];
    DevPlan &d = p->dp;
    d.rf_rings = f.rings;
    d.rf_n = (int)f.rings_h.size();
    d.rf_rest_smooth = f.rest_s;
    d.rf_n_rest_smooth = (int)f.rest_s_h.size();
    d.rf_rest_blue = f.rest_b;
    d.rf_n_rest_blue = (int)f.rest_b_h.size();
}

// Cost of one (ring, pair of maps) unit of the register-FFT ring kernel, for
// ordering its work: FFT work of length L = |rf_len|, twice for Bluestein
// rings and for the two rounds of length 4096; shorter transforms leave
// threads idle, so they count as 2048.
double rf_cost(int rf_len)
{
    const int L = std::abs(rf_len);
    if (L == 0) return 0.0;
    return (rf_len < 0 ? 2.0 : 1.0) * (L == 4096 ? 2.0 : 1.0) * std::max(L, 2048) * std::log2((double)L);
}

int build_tables(sht_plan_s *p, const Rings &R)
{
    const int L = p->lmax, M = p->mmax, nr = p->nrings;
    // ring pairs
    std::vector<double> px;
    std::vector<double> pss;
    std::vector<int2> pr;
    if (p->kind == SHT_GRID_RINGS) {
        for (int r = 0; r < nr; ++r) {
            px.push_back(R.x[r]);
            pss.push_back(R.s[r]);
            pr.push_back(make_int2(r, -1));
        }
    } else {
        for (int r = 0; r < nr / 2; ++r) {
            px.push_back(R.x[r]);
            pss.push_back(R.s[r]);
            pr.push_back(make_int2(r, nr - 1 - r));
        }
        if (nr % 2) {
            px.push_back(R.x[nr / 2]);
            pss.push_back(R.s[nr / 2]);
            pr.push_back(make_int2(nr / 2, -1));
        }
    }
    const int np = (int)px.size();
    p->npairs = np;

    // lambda_mm = mu_m sin^m(theta) (Eq. pmm with the Condon-Shortley sign),
    // carried as mantissa * 2^e and stored as (v, k): value = v * 2^(512 k)
    std::vector<double> fm(M + 1, 0.0);
    for (int m = 1; m <= M; ++m) fm[m] = -std::sqrt((2.0 * m + 1.0) / (2.0 * m));
    std::vector<double> sv((size_t)(M + 1) * np);
    std::vector<int> sk((size_t)(M + 1) * np);
    for (int q = 0; q < np; ++q) {
        const double s = pss[q];
        int e = 0;
        double v = std::frexp(1.0 / std::sqrt(4.0 * kPi), &e);
        for (int m = 0; m <= M; ++m) {
            if (m > 0) {
                v = v * s * fm[m];
                int de = 0;
                v = std::frexp(v, &de);
                e += de;
            }
            double vv;
            int kk;
            if (v == 0.0) {
                vv = 0.0;
                kk = 0;
            } else if (e > -sht::kScaleHi) {
                vv = std::ldexp(v, e);
                kk = 0;
            } else {
                // k = ceil((e - 256) / 512) < 0: the stored mantissa lies in [2^-257, 2^256)
                kk = (int)std::ceil((double)(e - sht::kScaleHi) / sht::kScaleUnit);
                vv = std::ldexp(v, e - sht::kScaleUnit * kk);
            }
            sv[(size_t)m * np + q] = vv;
            sk[(size_t)m * np + q] = kk;
        }
    }

    // scaled recurrence coefficients (see legendre_fp64.cu):
    // C_m = C_{m+1} = 1, C_l = (beta_l / beta_{l-1}) C_{l-2},
    // A_{m+1} = sqrt(2m+3), A_l = beta_{l-1} C_{l-1} / C_{l-2}
    std::vector<double> cA(p->nalm), cC(p->nalm);
    for (int m = 0; m <= M; ++m) {
        const long long o = mofs(L, m);
        auto beta = [m](int l) {
            const double dl = l, dm = m;
            return std::sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
        };
        cA[o] = 0.0;
        cC[o] = 1.0;
        if (m + 1 <= L) {
            cA[o + 1] = std::sqrt(2.0 * m + 3.0);
            cC[o + 1] = 1.0;
        }
        for (int l = m + 2; l <= L; ++l) {
            const double bl = beta(l), bl1 = beta(l - 1);
            cC[o + l - m] = (bl / bl1) * cC[o + l - m - 2];
            cA[o + l - m] = bl1 * cC[o + l - m - 1] / cC[o + l - m - 2];
        }
    }

    // rings and twiddle tables T_n[q] = e^{i pi q / n}, q < 2n
    std::vector<long long> ofs(nr);
    long long acc = 0;
    int maxn = 0, cap = 0;
    for (int r = 0; r < nr; ++r) {
        ofs[r] = acc;
        acc += R.nphi[r];
        maxn = std::max(maxn, R.nphi[r]);
        const int n = R.nphi[r];
        const int N = (n % 2 == 0) ? n / 2 : n;
        cap = std::max(cap, N + 1);
    }
    std::map<int, long long> where;
    std::vector<double2> tw64;
    std::vector<float2> tw32;
    std::vector<long long> twofs(nr);
    for (int r = 0; r < nr; ++r) {
        const int n = R.nphi[r];
        auto it = where.find(n);
        if (it == where.end()) {
            const long long o = (long long)tw64.size();
            where[n] = o;
            for (int q = 0; q < 2 * n; ++q) {
                const double a = kPi * (double)q / (double)n;
                const double c = std::cos(a), s = std::sin(a);
                tw64.push_back(make_double2(c, s));
                tw32.push_back(make_float2((float)c, (float)s));
            }
            twofs[r] = o;
        } else {
            twofs[r] = it->second;
        }
    }

    // both shared-memory FFT buffers of the FP64 ring kernel must fit in one CTA
    if (sht::ring_smem_bytes_for_cap(cap, true) > kMaxDynSmem)
        return fail(SHT_EUNSUPPORTED, "ring of %d pixels too long for the shared-memory FFT", maxn);

    // Bluestein rings and their chirp spectra
    std::vector<int> rsmooth, rblue, bmb(nr, 0);
    std::vector<long long> bofs(nr, -1);
    std::vector<double2> bh64;
    std::vector<float2> bh32;
    std::map<int, long long> bwhere;
    int bcap = 0;
    std::vector<long long> cofs(nr, 0);
    std::vector<float2> ch32;
    std::map<int, long long> cofs_of;
    for (int r = 0; r < nr; ++r) {
        const int n = R.nphi[r];
        const int N = (n % 2 == 0) ? n / 2 : n;
        int Mb = 1;
        while (Mb < 2 * N - 1) Mb <<= 1;
        if (largest_prime_factor(N) < sht::kBlueMinPrime || Mb > sht::kBlueMaxMb) {
            rsmooth.push_back(r);
            continue;
        }
        rblue.push_back(r);
        bmb[r] = Mb;
        bcap = std::max(bcap, Mb);
        auto it = bwhere.find(N);
        if (it != bwhere.end()) {
            bofs[r] = it->second;
            cofs[r] = cofs_of[N];
            continue;
        }
        const long long o = (long long)bh64.size();
        bwhere[N] = o;
        bofs[r] = o;
        cofs_of[N] = (long long)ch32.size();
        cofs[r] = cofs_of[N];
        for (int t = 0; t < N; ++t) {
            // c_t = e^{i pi t^2 / N}: the angle of the ring table's entry T_n[(t^2 mod 2N) n / N]
            const long long qn = (((long long)t * t) % (2LL * N)) * (n / N);
            const double a = kPi * (double)qn / (double)n;
            ch32.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
        }
        std::vector<double> re(Mb, 0.0), im(Mb, 0.0);
        for (int t = 0; t < N; ++t) {
            // b_t = e^{-i pi t^2 / N}, with t^2 reduced mod 2N for an exact angle
            const long long q = ((long long)t * t) % (2LL * N);
            const double a = -kPi * (double)q / (double)N;
            re[t] = std::cos(a);
            im[t] = std::sin(a);
            if (t > 0) {
                re[Mb - t] = re[t];
                im[Mb - t] = im[t];
            }
        }
        fft_pow2_forward(re, im);
        for (int k = 0; k < Mb; ++k) {
            bh64.push_back(make_double2(re[k] / Mb, im[k] / Mb));
            bh32.push_back(make_float2((float)(re[k] / Mb), (float)(im[k] / Mb)));
        }
    }
    // FP32 ring step with the FFT in registers: the ring's FFT length and, for
    // Bluestein rings, the chirp and chirp spectrum of that length (per distinct N)
    std::vector<int> rflen(nr, 0);
    std::vector<long long> rfco(nr, 0), rfbo(nr, 0);
    std::vector<float2> rfch, rfbh;
    std::map<int, std::pair<long long, long long>> rfwhere;
    const bool rf_fits = (size_t)2 * (((M + 1 + 255) / 256) * 256) * 16 + (size_t)(4096 + 256) * 8 <= kMaxDynSmem;
    for (int r = 0; r < nr && rf_fits; ++r) {
        const int n = R.nphi[r];
        if (n % 2) continue;
        const int N = n / 2;
        if ((N & (N - 1)) == 0 && N >= 256 && N <= 4096) {
            rflen[r] = N;
            continue;
        }
        if (N > 2048) continue;
        int Lb = 256;
        while (Lb < 2 * N - 1) Lb <<= 1;
        rflen[r] = -Lb;
        auto it = rfwhere.find(N);
        if (it != rfwhere.end()) {
            rfco[r] = it->second.first;
            rfbo[r] = it->second.second;
            continue;
        }
        rfco[r] = (long long)rfch.size();
        rfbo[r] = (long long)rfbh.size();
        rfwhere[N] = {rfco[r], rfbo[r]};
        for (int t = 0; t < N; ++t) {
            // c_t = e^{i pi t^2 / N}, t^2 reduced mod 2N for an exact angle
            const long long q = ((long long)t * t) % (2LL * N);
            const double a = kPi * (double)q / (double)N;
            rfch.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
        }
        std::vector<double> re(Lb, 0.0), im(Lb, 0.0);
        for (int t = 0; t < N; ++t) {
            const long long q = ((long long)t * t) % (2LL * N);
            const double a = -kPi * (double)q / (double)N;
            re[t] = std::cos(a);
            im[t] = std::sin(a);
            if (t > 0) {
                re[Lb - t] = re[t];
                im[Lb - t] = im[t];
            }
        }
        fft_pow2_forward(re, im);
        for (int k = 0; k < Lb; ++k) rfbh.push_back(make_float2((float)(re[k] / Lb), (float)(im[k] / Lb)));
    }
    // ring sets of the FP32 ring step per kernel choice (sht_debug_ring_kernel):
    // 0 (default): the register kernel runs the rings it transforms with
    // Bluestein's algorithm (N not a power of two), the shared-memory kernel the
    // others (measured at nside 1024, 64 maps: register kernel 4.5 ms for the
    // cap rings with a large prime factor against 6.1 ms, 2.0 ms against 3.0 ms
    // for the other non-power-of-two caps; shared-memory kernel 3.0 ms for the
    // equatorial belt against 3.2 ms); 1: shared-memory kernel for every ring;
    // 2: register kernel for every ring it can run
    std::vector<int> rfrings[3], rfrest_s[3], rfrest_b[3];
    for (int mode = 0; mode < 3; ++mode)
        for (int r = 0; r < nr; ++r) {
            bool reg = rflen[r] != 0 && mode != 1;
            if (mode == 0 && rflen[r] > 0) reg = false;
            if (reg) {
                rfrings[mode].push_back(r);
            } else if (bmb[r] > 0) {
                rfrest_b[mode].push_back(r);
            } else {
                rfrest_s[mode].push_back(r);
            }
        }
    // by decreasing cost, rings of equal cost kept in ring order
    for (auto &v : rfrings)
        std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return rf_cost(rflen[a]) > rf_cost(rflen[b]); });

    std::vector<double2> w2d(sht::kBlueMaxMb);
    std::vector<float2> w2f(sht::kBlueMaxMb);
    for (int q = 0; q < sht::kBlueMaxMb; ++q) {
        const double a = 2.0 * kPi * (double)q / sht::kBlueMaxMb;
        w2d[q] = make_double2(std::cos(a), std::sin(a));
        w2f[q] = make_float2((float)std::cos(a), (float)std::sin(a));
    }

    DevPlan &d = p->dp;
    d.lmax = L;
    d.mmax = M;
    d.nrings = nr;
    d.npairs = np;
    d.nalm = p->nalm;
    d.npix = p->npix;
    d.max_nphi = maxn;
    d.fft_cap = cap;
    int rc;
    if ((rc = upload(p, px, &d.pair_x))) return rc;
    if ((rc = upload(p, pr, &d.pair_ring))) return rc;
    p->pair_ring_h = pr;
    if ((rc = upload(p, sv, &d.start_v))) return rc;
    if ((rc = upload(p, sk, &d.start_k))) return rc;
    if ((rc = upload(p, cA, &d.coefA))) return rc;
    if ((rc = upload(p, cC, &d.coefC))) return rc;
    if ((rc = upload(p, R.nphi, &d.nphi))) return rc;
    if ((rc = upload(p, ofs, &d.ofs))) return rc;
    if ((rc = upload(p, R.phi0, &d.phi0))) return rc;
    if ((rc = upload(p, R.ps, &d.ps))) return rc;
    {
        // pixel quadrature weights: mutable (sht_set_ring_weights), zero when the grid has none
        p->wring_h = R.w.empty() ? std::vector<double>(nr, 0.0) : R.w;
        void *w = nullptr;
        cudaError_t e = cudaMalloc(&w, (size_t)nr * sizeof(double));
        if (e != cudaSuccess) return fail(SHT_ENOMEM, "cudaMalloc(weights): %s", cudaGetErrorString(e));
        p->allocs.push_back(w);
        e = cudaMemcpy(w, p->wring_h.data(), (size_t)nr * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(weights)");
        p->wring_d = static_cast<double *>(w);
        d.wring = p->wring_d;
    }
    if ((rc = upload(p, twofs, &d.twofs))) return rc;
    if ((rc = upload(p, tw64, &d.tw64))) return rc;
    if ((rc = upload(p, tw32, &d.tw32))) return rc;
    p->rings_smooth_h = rsmooth;
    p->nphi_h = R.nphi;
    p->min_sin = R.s.empty() ? 0.0 : *std::min_element(R.s.begin(), R.s.end());
    p->rings_blue_h = rblue;
    d.n_smooth = (int)rsmooth.size();
    d.n_blue = (int)rblue.size();
    d.blue_cap = bcap;
    if ((rc = upload(p, rsmooth, &d.rings_smooth))) return rc;
    if ((rc = upload(p, rblue, &d.rings_blue))) return rc;
    if ((rc = upload(p, bmb, &d.blue_mb))) return rc;
    if ((rc = upload(p, bofs, &d.blue_ofs))) return rc;
    if ((rc = upload(p, cofs, &d.chirp_ofs))) return rc;
    if ((rc = upload(p, ch32, &d.chirp32))) return rc;
    if ((rc = upload(p, bh64, &d.bhat64))) return rc;
    if ((rc = upload(p, bh32, &d.bhat32))) return rc;
    if ((rc = upload(p, w2d, &d.w2_64))) return rc;
    if ((rc = upload(p, w2f, &d.w2_32))) return rc;
    if ((rc = upload(p, rflen, &d.rf_len))) return rc;
    if ((rc = upload(p, rfco, &d.rf_ch_ofs))) return rc;
    if ((rc = upload(p, rfbo, &d.rf_bh_ofs))) return rc;
    if ((rc = upload(p, rfch, &d.rf_ch32))) return rc;
    if ((rc = upload(p, rfbh, &d.rf_bh32))) return rc;
    for (int mode = 0; mode < 3; ++mode) {
        auto &f = p->rf_set[mode];
        if ((rc = upload(p, rfrings[mode], &f.rings)) || (rc = upload(p, rfrest_s[mode], &f.rest_s)) ||
            (rc = upload(p, rfrest_b[mode], &f.rest_b)))
            return rc;
        f.rings_h = rfrings[mode];
        f.rest_s_h = rfrest_s[mode];
        f.rest_b_h = rfrest_b[mode];
    }
    p->rf_len_h = rflen;
    apply_rf_mode(p);

    // tensor-core forms: (m, parity) segments of the B operand, padded to
    // whole stages of KC degrees per parity (KC = 8 for TF32, 16 for BF16)
    for (int pass = 0; pass < 2; ++pass) {
        const int kc = pass == 0 ? 8 : 16;
        std::vector<int> seg(2 * (size_t)(M + 1));
        long long off = 0;
        for (int m = 0; m <= M; ++m) {
            const long long kpad = (long long)((L - m + 1 + 2 * kc - 1) / (2 * kc)) * kc;
            seg[2 * m] = (int)off;
            off += kpad;
            seg[2 * m + 1] = (int)off;
            off += kpad;
        }
        if (off > 0x7fffffffLL) return fail(SHT_EUNSUPPORTED, "tensor-core operand too large");
        if (pass == 0) {
            if ((rc = upload(p, seg, &p->tc.seg_tf32))) return rc;
            p->tc.kall_tf32 = off;
        } else {
            if ((rc = upload(p, seg, &p->tc.seg_bf16))) return rc;
            p->tc.kall_bf16 = off;
        }
    }
#ifdef SHT_DEBUG
    {
        // debug words of the kernels' index checks (count, first tag, index, bound)
        void *w = nullptr;
        cudaError_t e = cudaMalloc(&w, 4 * sizeof(unsigned long long));
        if (e != cudaSuccess) return fail(SHT_ENOMEM, "cudaMalloc(debug words): %s", cudaGetErrorString(e));
        p->allocs.push_back(w);
        if ((e = cudaMemset(w, 0, 4 * sizeof(unsigned long long))) != cudaSuccess) return cuda_fail(e, "cudaMemset");
        d.dbg = static_cast<unsigned long long *>(w);
    }
#endif
    {
        void *st = nullptr;
        cudaError_t e = cudaMalloc(&st, sizeof(int));
        if (e != cudaSuccess) return fail(SHT_ENOMEM, "cudaMalloc(status): %s", cudaGetErrorString(e));
        p->allocs.push_back(st);
        e = cudaMemset(st, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
        p->tc.status = static_cast<int *>(st);
    }
    return SHT_OK;
}

// Grow the Delta workspace to at least `bytes` (stream-ordered callers only).
int ensure_ws(sht_plan_s *p, size_t bytes)
{
    if (p->ws_bytes >= bytes) return SHT_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    if (p->ws) cudaFree(p->ws);
    p->ws = nullptr;
    p->ws_bytes = 0;
    e = cudaMalloc(&p->ws, bytes);
    if (e != cudaSuccess) {
        p->ws = nullptr;
        cudaGetLastError();
        return fail(SHT_ENOMEM, "workspace cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    p->ws_bytes = bytes;
    return SHT_OK;
}

int ensure_tc(sht_plan_s *p, int prec)
{
    const size_t need = sht::tc_bbuf_bytes(p->tc, prec);
    if (p->tc_bytes >= need) return SHT_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    if (p->tc.bbuf) cudaFree(p->tc.bbuf);
    p->tc.bbuf = nullptr;
    p->tc_bytes = 0;
    e = cudaMalloc(&p->tc.bbuf, need);
    if (e != cudaSuccess) {
        p->tc.bbuf = nullptr;
        cudaGetLastError();
        return fail(SHT_ENOMEM, "tensor-core operand cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
    }
    p->tc_bytes = need;
    return SHT_OK;
}

size_t max_ws_bytes()
{
    const char *env = std::getenv("SHT_MAX_WORKSPACE_MB");
    if (env) {
        const long long v = std::atoll(env);
        if (v > 0) return (size_t)v << 20;
    }
    return (size_t)16 << 30;
}

int check_plan(sht_plan_t p)
{
    if (!p) return fail(SHT_EINVAL, "null plan");
    return SHT_OK;
}

// Cost share of a tensor-core work item's setup and Delta epilogue, in degrees
// of its recurrence (fitted to per-CTA clock counts: about 1.5 stages).
constexpr long long kItemOverhead = 48;

// Work lists of a persistent launch: the items, in the order given, go one by
// one to the list with the least cost so far (ties: the lowest list index),
// which replays a work queue served in that order.  List b is items[off[b] ..
// off[b + 1]), in serving order; off has nlists + 1 entries.
void build_work_lists(int nitems, const long long *cost, int nlists, int *off, int *items)
{
    using Slot = std::pair<long long, int>;  // (cost so far, list)
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> q;
    for (int b = 0; b < nlists; ++b) q.push({0, b});
    std::vector<int> owner((size_t)nitems);
    std::fill(off, off + nlists + 1, 0);
    for (int j = 0; j < nitems; ++j) {
        const Slot t = q.top();
        q.pop();
        owner[j] = t.second;
        ++off[t.second + 1];
        q.push({t.first + cost[j], t.second});
    }
    for (int b = 0; b < nlists; ++b) off[b + 1] += off[b];
    std::vector<int> fill(off, off + nlists);
    for (int j = 0; j < nitems; ++j) items[fill[owner[j]]++] = j;
}

// The work lists of the persistent tensor-core launches for the plan's current
// skip tables: items served in m order (ring block minor).  The cost of an
// item is the degrees its recurrence runs plus a fixed share for its setup and
// Delta epilogue.
int ensure_sched(sht_plan_s *p, cudaStream_t st)
{
    sht::DevPlan &d = p->dp;
    const int want = d.skip_g ? 1 : 0;
    const int nrb = (p->npairs + 127) / 128;
    const int nitems = nrb * (p->mmax + 1);
    if (p->sched_off) {
        d.sched_ctas = 0;
        return SHT_OK;
    }
    if (p->sched && p->sched_skip == want) {
        d.sched_off = p->sched;
        d.sched_items = p->sched + d.sched_ctas + 1;
        return SHT_OK;
    }
    d.sched_ctas = 0;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "work lists");
    const int G = std::min(nitems, nsm);
    std::vector<int> g0((size_t)nitems, 0);
    if (d.skip_g) {
        e = cudaMemcpyAsync(g0.data(), d.skip_g, (size_t)nitems * sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "work lists");
    }
    // items past every ring of their block (Delta exactly zero there) are left out
    const bool cut = d.skip_g && d.ring_mlim && (int)p->blim_h.size() == nrb;
    std::vector<int> keep;
    std::vector<long long> cost;
    for (int j = 0; j < nitems; ++j) {
        if (cut && j / nrb >= p->blim_h[j % nrb]) continue;
        keep.push_back(j);
        cost.push_back((p->lmax - j / nrb + 1 - 64LL * g0[j]) + kItemOverhead);
    }
    const int nkept = (int)keep.size();
    std::vector<int> host((size_t)G + 1 + nkept, 0);
    build_work_lists(nkept, cost.data(), G, host.data(), host.data() + G + 1);
    for (int j = 0; j < nkept; ++j) host[G + 1 + j] = keep[host[G + 1 + j]];
    if (!p->sched) {
        // sized for every item: the lists of the other skip setting reuse it
        e = cudaMalloc(&p->sched, ((size_t)G + 1 + nitems) * sizeof(int));
        if (e != cudaSuccess) {
            p->sched = nullptr;
            cudaGetLastError();
            return fail(SHT_ENOMEM, "work lists: %s", cudaGetErrorString(e));
        }
    }
    e = cudaMemcpyAsync(p->sched, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "work lists");
    p->sched_skip = want;
    d.sched_ctas = G;
    d.sched_off = p->sched;
    d.sched_items = p->sched + G + 1;
    return SHT_OK;
}

// Evanescent-skip tables of the tensor-core forms: built on first use (one
// FP64 pass over the recurrence, synchronous), or detached when disabled; then
// the work lists for that setting.  The same pass gives each ring the orders
// at which its Delta can be nonzero (DevPlan::ring_mlim) and each ring block
// the largest of them (blim_h), past which the block's items are left out.
int ensure_warm(sht_plan_s *p, cudaStream_t st)
{
    sht::DevPlan &d = p->dp;
    if (!p->skip_evanescent) {
        d.skip_g = nullptr;
        d.warm_p0 = d.warm_p1 = nullptr;
        d.warm_k = nullptr;
        d.ring_mlim = nullptr;
        d.block_mlim = nullptr;
        return ensure_sched(p, st);
    }
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t nrb = (size_t)((p->npairs + 127) / 128), M1 = (size_t)p->mmax + 1;
    const size_t nst = M1 * (size_t)p->npairs;
    const size_t b_g = up(M1 * nrb * sizeof(int));
    const size_t b_p = nst * sizeof(double);
    const size_t o_k = b_g + 2 * b_p;
    const size_t o_lim = o_k + up(nst * sizeof(int));
    const size_t o_rl = o_lim + up((size_t)p->npairs * sizeof(int));
    const size_t o_bl = o_rl + up((size_t)p->nrings * sizeof(int));
    const size_t total = o_bl + nrb * sizeof(int);
    if (!p->warm) {
        cudaError_t e = cudaMalloc(&p->warm, total);
        if (e != cudaSuccess) {
            p->warm = nullptr;
            cudaGetLastError();
            return fail(SHT_ENOMEM, "skip tables: %s", cudaGetErrorString(e));
        }
        char *b = static_cast<char *>(p->warm);
        int *g = reinterpret_cast<int *>(b);
        double *w0 = reinterpret_cast<double *>(b + b_g), *w1 = reinterpret_cast<double *>(b + b_g + b_p);
        int *wk = reinterpret_cast<int *>(b + o_k);
        int *plim = reinterpret_cast<int *>(b + o_lim);
        d.skip_g = nullptr;  // the build itself starts every item at degree m
        d.ring_mlim = nullptr;
        d.block_mlim = nullptr;
        e = cudaMemsetAsync(plim, 0, (size_t)p->npairs * sizeof(int), st);
        if (e == cudaSuccess) e = sht::launch_warm_start(d, g, w0, w1, wk, plim, st);
        if (e == cudaSuccess) {
            g_launches.fetch_add(1, std::memory_order_relaxed);
            e = cudaStreamSynchronize(st);
        }
        // per ring: its pair's limit; per ring block: the largest over its pairs
        std::vector<int> pl((size_t)p->npairs), rl((size_t)p->nrings, 0);
        if (e == cudaSuccess)
            e = cudaMemcpy(pl.data(), plim, pl.size() * sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            p->blim_h.assign(nrb, 1);
            for (int q = 0; q < p->npairs; ++q) {
                const int lim = std::min(std::max(pl[q], 1), p->mmax + 1);
                const int2 rr = p->pair_ring_h[q];
                rl[rr.x] = lim;
                if (rr.y >= 0) rl[rr.y] = lim;
                int &bl = p->blim_h[q / 128];
                bl = std::max(bl, lim);
            }
            e = cudaMemcpy(b + o_rl, rl.data(), rl.size() * sizeof(int), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(b + o_bl, p->blim_h.data(), p->blim_h.size() * sizeof(int), cudaMemcpyHostToDevice);
            p->ring_mlim_h = rl;
        }
        if (e != cudaSuccess) {
            cudaFree(p->warm);
            p->warm = nullptr;
            p->blim_h.clear();
            return cuda_fail(e, "warm_start");
        }
    }
    char *b = static_cast<char *>(p->warm);
    d.skip_g = reinterpret_cast<const int *>(b);
    d.warm_p0 = reinterpret_cast<const double *>(b + b_g);
    d.warm_p1 = reinterpret_cast<const double *>(b + b_g + b_p);
    d.warm_k = reinterpret_cast<const int *>(b + o_k);
    d.ring_mlim = reinterpret_cast<const int *>(b + o_rl);
    d.block_mlim = reinterpret_cast<const int *>(b + o_bl);
    return ensure_sched(p, st);
}

double rf_unit_cost(const sht_plan_s *p, int r) { return rf_cost(p->rf_len_h[r]); }

// FP32 ring step of the tensor-core forms: the register-FFT kernel over the
// plan's rf_rings, then the shared-memory kernel over the other rings (odd
// lengths, long rings without a power-of-two transform); *nk = kernels launched.
cudaError_t ring_step_fp32(sht_plan_s *p, const float2 *delta, float *map, int nb, cudaStream_t st, int *nk)
{
    *nk = 0;
    cudaError_t e = sht::launch_ring_reg(p->dp, delta, map, nb, p->tc.status, st);
    if (e != cudaSuccess) return e;
    *nk += p->dp.rf_n > 0;
    if (p->dp.rf_n_rest_smooth + p->dp.rf_n_rest_blue == 0) return cudaSuccess;
    DevPlan q = p->dp;
    q.rings_smooth = q.rf_rest_smooth;
    q.n_smooth = q.rf_n_rest_smooth;
    q.rings_blue = q.rf_rest_blue;
    q.n_blue = q.rf_n_rest_blue;
    e = sht::launch_ring_synth_mf(q, delta, map, nb, p->ring_g[0], p->ring_g[1], p->ring_nt, st);
    *nk += sht::ring_launches(q);
    return e;
}

// Precision forms: FP64 recurrence (or the plan-time Lambda operand, when
// cached) + tensor-core contraction (groups of at most 64 maps), FP32 Delta,
// FP32 ring step, float32 maps.
int alm2map_tc(sht_plan_s *p, int nbatch, const void *alm_dev, void *map_dev, int prec, void *stream)
{
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard dg(p->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc;
    const int group = std::min(nbatch, sht::kTcMaxMaps);
    const size_t per_map = (size_t)p->nrings * (p->mmax + 1) * sizeof(float2);
    if ((rc = ensure_ws(p, per_map * group))) return rc;
    if ((rc = ensure_tc(p, prec))) return rc;
    if ((rc = ensure_warm(p, st))) return rc;
    const double2 *alm = static_cast<const double2 *>(alm_dev);
    float *map = static_cast<float *>(map_dev);
    float2 *delta = static_cast<float2 *>(p->ws);  // [ring][m][map]
    for (int b0 = 0; b0 < nbatch; b0 += group) {
        const int nb = std::min(group, nbatch - b0);
        StageScope s0(p, SHT_STAGE_OPERAND_PREP, st);
        cudaError_t e = sht::launch_tc_prep(p->dp, p->tc, prec, alm + (size_t)b0 * p->nalm, nb, st);
        s0.done(e);
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core operand prep launch");
        StageScope s1(p, SHT_STAGE_LEGENDRE, st);
        e = sht::launch_tc_main(p->dp, p->tc, prec, p->lcache[prec], delta, nb, st);
        p->tc.withhold = -1;  // the test hook applies to one launch
        s1.done(e);
        if (e != cudaSuccess) return cuda_fail(e, "legendre_tc launch");
        StageScope s2(p, SHT_STAGE_RING, st);
        int nk = 0;
        e = ring_step_fp32(p, delta, map + (size_t)b0 * p->npix, nb, st, &nk);
        s2.done(e, nk);
        if (e != cudaSuccess) return cuda_fail(e, "FP32 ring step launch");
    }
    return SHT_OK;
}

// FP64 alm2map of nbatch maps (caller holds the plan lock and the device).
int alm2map_fp64(sht_plan_s *p, int nbatch, const double2 *alm, double *map, cudaStream_t st)
{
    int rc;
    const size_t per_map = (size_t)p->nrings * (p->mmax + 1) * sizeof(double2);
    size_t chunk_sz = std::max<size_t>(1, max_ws_bytes() / per_map);
    int chunk = (int)std::min<size_t>(chunk_sz, 32768);  // grid.y limit of the ring kernel
    chunk = std::min(chunk, nbatch);
    if ((rc = ensure_ws(p, per_map * chunk))) return rc;
    double2 *delta = static_cast<double2 *>(p->ws);
    for (int b0 = 0; b0 < nbatch; b0 += chunk) {
        const int nb = std::min(chunk, nbatch - b0);
        StageScope s1(p, SHT_STAGE_LEGENDRE, st);
        cudaError_t e = sht::launch_legendre_fwd_fp64(p->dp, alm + (size_t)b0 * p->nalm, delta, nb, p->fp64_bc, st);
        s1.done(e);
        if (e != cudaSuccess) return cuda_fail(e, "legendre_fwd_fp64 launch");
        StageScope s2(p, SHT_STAGE_RING, st);
        e = sht::launch_ring_synth_fp64(p->dp, delta, map + (size_t)b0 * p->npix, nb, p->fp64_ring_g, st);
        s2.done(e, sht::ring_launches(p->dp));
        if (e != cudaSuccess) return cuda_fail(e, "ring_synth_fp64 launch");
    }
    return SHT_OK;
}

// Quadrature-weighted ring analysis + Legendre sum (weights from the plan) or
// the plain transpose (weights nullptr, cfac 2) of nbatch FP64 maps (caller
// holds the plan lock and the device).
int analysis_fp64(sht_plan_s *p, int nbatch, const double *map, double2 *alm, const double *wring, double cfac,
                  cudaStream_t st)
{
    int rc;
    const size_t per_map = (size_t)p->nrings * (p->mmax + 1) * sizeof(double2);
    size_t chunk_sz = std::max<size_t>(1, max_ws_bytes() / per_map);
    int chunk = (int)std::min<size_t>(chunk_sz, 32768);
    chunk = std::min(chunk, nbatch);
    if ((rc = ensure_ws(p, per_map * chunk))) return rc;
    double2 *q = static_cast<double2 *>(p->ws);
    for (int b0 = 0; b0 < nbatch; b0 += chunk) {
        const int nb = std::min(chunk, nbatch - b0);
        StageScope s1(p, SHT_STAGE_ADJ_RING, st);
        cudaError_t e = sht::launch_ring_analysis_fp64(p->dp, map + (size_t)b0 * p->npix, q, nb, wring, st);
        s1.done(e, sht::ring_launches(p->dp));
        if (e != cudaSuccess) return cuda_fail(e, "ring_analysis_fp64 launch");
        StageScope s2(p, SHT_STAGE_ADJ_LEGENDRE, st);
        e = sht::launch_legendre_adj_fp64(p->dp, q, alm + (size_t)b0 * p->nalm, nb, cfac, st);
        s2.done(e);
        if (e != cudaSuccess) return cuda_fail(e, "legendre_adj_fp64 launch");
    }
    return SHT_OK;
}

// The transpose in a BF16 tensor-core form (caller holds the plan lock and
// the device): FP32 ring analysis of groups of up to 32 float maps, then the
// contraction from the plan-time Lambda operand of that form, which must have
// been built (sht_lambda_cache).  Weights and cfac as analysis_fp64.
int analysis_tc(sht_plan_s *p, int nbatch, const float *map, double2 *alm, const double *wring, double cfac,
                int prec, cudaStream_t st)
{
    int rc;
    if (prec != SHT_BF16X3_TC && prec != SHT_BF16X6_TC)
        return fail(SHT_EUNSUPPORTED, "the transpose has no tensor-core form for precision %d (BF16 forms only)", prec);
    if (!p->lcache[prec])
        return fail(SHT_EUNSUPPORTED,
                    "the tensor-core transpose reads the plan-time Lambda operand: build it first (sht_lambda_cache)");
    if ((rc = ensure_tc(p, prec)) || (rc = ensure_warm(p, st))) return rc;
    constexpr int G = 32;  // maps per contraction launch
    const size_t qb = (size_t)G * p->nrings * (p->mmax + 1) * sizeof(float2);
    const size_t need = qb + sht::adj_tc_bimg_bytes(p->dp, prec, G);
    if (p->adj_bytes < need) {
        if (p->adj_ws) {
            cudaError_t e = cudaDeviceSynchronize();  // an earlier call may still use it
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
            cudaFree(p->adj_ws);
        }
        p->adj_ws = nullptr;
        p->adj_bytes = 0;
        cudaError_t e = cudaMalloc(&p->adj_ws, need);
        if (e != cudaSuccess) {
            p->adj_ws = nullptr;
            cudaGetLastError();
            return fail(SHT_ENOMEM, "transpose workspace: %s", cudaGetErrorString(e));
        }
        p->adj_bytes = need;
    }
    if (!p->adj_items) {
        std::vector<int2> it;
        for (int m = 0; m <= p->mmax; ++m) {
            const int nst = (p->lmax - m + 1 + 31) / 32;
            for (int j = 0; j < (nst + 7) / 8; ++j) it.push_back(make_int2(m, j));
        }
        cudaError_t e = cudaMalloc(&p->adj_items, it.size() * sizeof(int2));
        if (e == cudaSuccess)
            e = cudaMemcpy(p->adj_items, it.data(), it.size() * sizeof(int2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (p->adj_items) cudaFree(p->adj_items);
            p->adj_items = nullptr;
            cudaGetLastError();
            return fail(SHT_ENOMEM, "transpose items: %s", cudaGetErrorString(e));
        }
        p->adj_nitems = (int)it.size();
    }
    float2 *q = static_cast<float2 *>(p->adj_ws);
    void *bimg = static_cast<char *>(p->adj_ws) + qb;
    for (int b0 = 0; b0 < nbatch; b0 += G) {
        const int nb = std::min(G, nbatch - b0);
        StageScope s1(p, SHT_STAGE_ADJ_RING, st);
        cudaError_t e =
            sht::launch_ring_analysis_fp32(p->dp, map + (size_t)b0 * p->npix, q, nb, wring, p->adj_ring_g, st);
        s1.done(e, sht::ring_launches(p->dp));
        if (e != cudaSuccess) return cuda_fail(e, "ring_analysis_fp32 launch");
        StageScope s2(p, SHT_STAGE_ADJ_LEGENDRE, st);
        e = sht::launch_adj_tc(p->dp, p->tc, prec, p->lcache[prec], q, bimg, p->adj_items, p->adj_nitems,
                               alm + (size_t)b0 * p->nalm, nb, cfac, st);
        s2.done(e, 2);
        if (e != cudaSuccess) return cuda_fail(e, "legendre_adj_tc launch");
    }
    return SHT_OK;
}

// Jacobi refinement helpers: r = y - s (in place in s), a += d.
__global__ void residual_kernel(const double *__restrict__ y, double *__restrict__ s, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s[i] = y[i] - s[i];
}
__global__ void accumulate_kernel(double2 *__restrict__ a, const double2 *__restrict__ d, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        a[i].x += d[i].x;
        a[i].y += d[i].y;
    }
}

}  // namespace

extern "C" {

const char *sht_last_error(void) { return g_err.c_str(); }

int sht_plan(const sht_grid *g, int lmax, int mmax, sht_plan_t *out)
{
    g_err.clear();
    if (!out) return fail(SHT_EINVAL, "null output pointer");
    *out = nullptr;
    if (!g) return fail(SHT_EINVAL, "null grid");
    if (lmax < 0 || mmax < 0 || mmax > lmax) return fail(SHT_EINVAL, "need 0 <= mmax <= lmax");
    if (lmax > kMaxL) return fail(SHT_EUNSUPPORTED, "lmax > %d", kMaxL);
    Rings R;
    switch (g->kind) {
    case SHT_GRID_GL:
        if (g->nrings < 1 || g->nphi_gl < 1) return fail(SHT_EINVAL, "GL grid needs nrings, nphi_gl >= 1");
        if (g->nphi_gl > kMaxNphi) return fail(SHT_EUNSUPPORTED, "nphi > %d", kMaxNphi);
        if (g->nrings > 65536) return fail(SHT_EUNSUPPORTED, "too many rings");
        gl_geometry(g->nrings, g->nphi_gl, R);
        break;
    case SHT_GRID_HEALPIX:
        if (g->nside < 1) return fail(SHT_EINVAL, "HEALPix grid needs nside >= 1");
        if (4 * (long long)g->nside > kMaxNphi) return fail(SHT_EUNSUPPORTED, "nside > %d", kMaxNphi / 4);
        healpix_geometry(g->nside, R);
        break;
    case SHT_GRID_RINGS: {
        if (g->nrings < 1 || !g->theta || !g->nphi || !g->phi0)
            return fail(SHT_EINVAL, "RINGS grid needs nrings >= 1 and theta, nphi, phi0");
        if (g->nrings > 65536) return fail(SHT_EUNSUPPORTED, "too many rings");
        const int n = g->nrings;
        R.x.resize(n);
        R.s.resize(n);
        R.nphi.resize(n);
        R.phi0.resize(n);
        R.ps.resize(n);
        for (int r = 0; r < n; ++r) {
            const double th = g->theta[r];
            if (!(th >= 0.0 && th <= kPi)) return fail(SHT_EINVAL, "theta[%d] outside [0, pi]", r);
            if (g->nphi[r] < 1) return fail(SHT_EINVAL, "nphi[%d] < 1", r);
            if (g->nphi[r] > kMaxNphi) return fail(SHT_EUNSUPPORTED, "nphi[%d] > %d", r, kMaxNphi);
            if (!std::isfinite(g->phi0[r])) return fail(SHT_EINVAL, "phi0[%d] not finite", r);
            R.x[r] = std::cos(th);
            R.s[r] = std::sin(th);
            R.nphi[r] = g->nphi[r];
            R.phi0[r] = g->phi0[r];
            R.ps[r] = (g->phi0[r] == 0.0) ? 0 : -1;
        }
        break;
    }
    default:
        return fail(SHT_EINVAL, "unknown grid kind %d", g->kind);
    }

    auto *p = new (std::nothrow) sht_plan_s();
    if (!p) return fail(SHT_ENOMEM, "plan allocation");
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaGetDevice");
    }
    p->kind = g->kind;
    p->lmax = lmax;
    p->mmax = mmax;
    p->nrings = (int)R.x.size();
    p->nalm = (long long)(mmax + 1) * (2LL * lmax + 2 - mmax) / 2;
    long long npix = 0;
    for (int v : R.nphi) npix += v;
    p->npix = npix;
    int rc = build_tables(p, R);
    if (rc != SHT_OK) {
        std::string keep = g_err;
        free_plan(p);
        g_err = keep;
        return rc;
    }
    *out = p;
    return SHT_OK;
}

long long sht_lambda_cache_bytes(sht_plan_t p, int prec)
{
    if (!p || (prec != SHT_FP32_TC && prec != SHT_BF16X3_TC && prec != SHT_BF16X6_TC)) return 0;
    return (long long)sht::tc_lambda_bytes(p->dp, p->tc, prec);
}

int sht_lambda_cache(sht_plan_t p, int prec, int enable, void *stream)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (prec != SHT_FP32_TC && prec != SHT_BF16X3_TC && prec != SHT_BF16X6_TC)
        return fail(SHT_EINVAL, "the Lambda operand exists for the tensor-core forms only (prec %d)", prec);
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard dg(p->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!enable) {
        if (!p->lcache[prec]) return SHT_OK;
        cudaError_t e = cudaDeviceSynchronize();  // no launch may still read it
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
        cudaFree(p->lcache[prec]);
        p->lcache[prec] = nullptr;
        p->lcache_bytes[prec] = 0;
        return SHT_OK;
    }
    if (p->lcache[prec]) return SHT_OK;
    if ((rc = ensure_warm(p, st))) return rc;
    const size_t need = sht::tc_lambda_bytes(p->dp, p->tc, prec);
    void *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SHT_ENOMEM, "Lambda operand cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
    }
    // zero first: the stages the evanescent skip leaves unwritten hold exact
    // zeros, so the operand is valid with the skip on or off
    e = cudaMemsetAsync(buf, 0, need, st);
    if (e == cudaSuccess) e = sht::launch_lambda_build(p->dp, p->tc, prec, buf, st);
    if (e == cudaSuccess) {
        g_launches.fetch_add(1, std::memory_order_relaxed);
        e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
        cudaFree(buf);
        return cuda_fail(e, "lambda_build");
    }
    p->lcache[prec] = buf;
    p->lcache_bytes[prec] = need;
    return SHT_OK;
}

int sht_autotune(sht_plan_t p, int prec, int nbatch, void *stream)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (prec != SHT_FP64 && prec != SHT_FP32_TC && prec != SHT_BF16X3_TC && prec != SHT_BF16X6_TC)
        return fail(SHT_EINVAL, "unknown precision %d", prec);
    if (nbatch < 1) return fail(SHT_EINVAL, "nbatch < 1");
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard dg(p->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool tc = prec != SHT_FP64;
    // the launch group the transforms use: up to 64 maps (tensor-core forms), up to 8 for the
    // FP64 Legendre candidates (each runs the full recurrence and contraction)
    const int nb = std::min(nbatch, tc ? sht::kTcMaxMaps : 64);
    const size_t esz = tc ? sizeof(float2) : sizeof(double2);
    const size_t per_map = (size_t)p->nrings * (p->mmax + 1) * esz;
    if ((rc = ensure_ws(p, per_map * nb))) return rc;
    void *map = nullptr, *alm = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (map) cudaFree(map);
        if (alm) cudaFree(alm);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&map, (size_t)nb * p->npix * (tc ? sizeof(float) : sizeof(double)));
    if (e == cudaSuccess) e = cudaMemsetAsync(p->ws, 0, per_map * nb, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SHT_ENOMEM : SHT_ECUDA, "autotune set-up: %s",
                    cudaGetErrorString(e));
    }
    // one untimed launch, then `reps` timed ones; +inf on a launch error
    auto time_it = [&](auto launch, int reps) -> float {
        if (launch() != cudaSuccess) {
            cudaGetLastError();
            return 3.4e38f;
        }
        cudaEventRecord(e0, st);
        for (int i = 0; i < reps; ++i)
            if (launch() != cudaSuccess) {
                cudaGetLastError();
                return 3.4e38f;
            }
        cudaEventRecord(e1, st);
        float ms = 3.4e38f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            return 3.4e38f;
        }
        return ms;
    };
    if (tc) {
        // FP32 ring step: maps per CTA for the two ring lists x threads per CTA of
        // the shared-memory kernel, on the rings it runs (those outside rf_rings)
        const float2 *d = static_cast<const float2 *>(p->ws);
        DevPlan q = p->dp;
        q.rings_smooth = q.rf_rest_smooth;
        q.n_smooth = q.rf_n_rest_smooth;
        q.rings_blue = q.rf_rest_blue;
        q.n_blue = q.rf_n_rest_blue;
        float best = 3.4e38f;
        int bs = p->ring_g[0], bb = p->ring_g[1], bt = p->ring_nt;
        for (int nt : {256, 512})
            if (q.n_smooth + q.n_blue > 0)
            for (int gsm : {1, 2, 4})
                for (int gbl : {1, 2}) {
                    const float ms = time_it(
                        [&]() {
                            return sht::launch_ring_synth_mf(q, d, static_cast<float *>(map), nb, gsm, gbl, nt, st);
                        },
                        2);
                    if (ms < best) {
                        best = ms;
                        bs = gsm;
                        bb = gbl;
                        bt = nt;
                    }
                }
        p->ring_g[0] = bs;
        p->ring_g[1] = bb;
        p->ring_nt = bt;
    } else {
        const int nl = std::min(nb, 8);
        e = cudaMalloc(&alm, (size_t)nl * p->nalm * sizeof(double2));
        if (e == cudaSuccess) e = cudaMemsetAsync(alm, 0, (size_t)nl * p->nalm * sizeof(double2), st);
        if (e != cudaSuccess) {
            cleanup();
            cudaGetLastError();
            return fail(SHT_ENOMEM, "autotune set-up: %s", cudaGetErrorString(e));
        }
        float best = 3.4e38f;
        int bbc = p->fp64_bc;
        for (int bc : {1, 2, 4, 8}) {
            if (bc > nl) break;
            const float ms = time_it(
                [&]() {
                    return sht::launch_legendre_fwd_fp64(p->dp, static_cast<const double2 *>(alm),
                                                         static_cast<double2 *>(p->ws), nl, bc, st);
                },
                1);
            if (ms < best) {
                best = ms;
                bbc = bc;
            }
        }
        p->fp64_bc = bbc;
        best = 3.4e38f;
        int bg = p->fp64_ring_g;
        for (int g : {2, 4, 8, 16}) {
            if (g > nb && g > 2) break;
            const float ms = time_it(
                [&]() {
                    return sht::launch_ring_synth_fp64(p->dp, static_cast<const double2 *>(p->ws),
                                                       static_cast<double *>(map), nb, g, st);
                },
                2);
            if (ms < best) {
                best = ms;
                bg = g;
            }
        }
        p->fp64_ring_g = bg;
    }
    cleanup();
    return SHT_OK;
}

int sht_tiles(sht_plan_t p, int *out, int n)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (!out || n < 0) return fail(SHT_EINVAL, "null output or n < 0");
    const int v[6] = {p->ring_g[0], p->ring_g[1], p->ring_nt, p->fp64_bc, p->fp64_ring_g, p->adj_ring_g};
    for (int i = 0; i < n && i < 6; ++i) out[i] = v[i];
    return SHT_OK;
}

int sht_skip_evanescent(sht_plan_t p, int enable)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(p->mu);
    p->skip_evanescent = enable != 0;
    return SHT_OK;
}

int sht_work_lists(int nitems, const long long *cost, int nlists, int *off, int *items)
{
    if (nitems < 0 || nlists < 1 || !off || (nitems > 0 && (!cost || !items)))
        return fail(SHT_EINVAL, "sht_work_lists: bad arguments");
    for (int j = 0; j < nitems; ++j)
        if (cost[j] < 0) return fail(SHT_EINVAL, "sht_work_lists: negative cost of item %d", j);
    build_work_lists(nitems, cost, nlists, off, items);
    return SHT_OK;
}

int sht_debug_work_lists(sht_plan_t p, int enable)
{
    if (!p) return fail(SHT_EINVAL, "sht_debug_work_lists: NULL plan");
    std::lock_guard<std::mutex> lk(p->mu);
    p->sched_off = !enable;
    return SHT_OK;
}

int sht_debug_report(sht_plan_t p, unsigned long long *out)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (!out) return fail(SHT_EINVAL, "null output array");
    out[0] = out[1] = out[2] = out[3] = out[4] = 0;
#ifdef SHT_DEBUG
    out[0] = 1;
    DeviceGuard dg(p->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(out + 1, p->dp.dbg, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p->dp.dbg, 0, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e, "debug words");
#endif
    return SHT_OK;
}

int sht_debug_ring_kernel(sht_plan_t p, int mode)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (mode < 0 || mode > 2) return fail(SHT_EINVAL, "ring kernel choice %d not in 0..2", mode);
    std::lock_guard<std::mutex> lk(p->mu);
    p->rf_mode = mode;
    apply_rf_mode(p);
    return SHT_OK;
}

int sht_order_limits(sht_plan_t p, int *out)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (!out) return fail(SHT_EINVAL, "null output array");
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard dg(p->device);
    if (p->skip_evanescent && (rc = ensure_warm(p, nullptr))) return rc;
    for (int r = 0; r < p->nrings; ++r)
        out[r] = p->skip_evanescent && !p->ring_mlim_h.empty() ? p->ring_mlim_h[r] : p->mmax + 1;
    return SHT_OK;
}

int sht_debug_poison_delta(sht_plan_t p)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard dg(p->device);
    if (!p->ws) return SHT_OK;
    cudaError_t e = cudaMemset(p->ws, 0xFF, p->ws_bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? SHT_OK : cuda_fail(e, "poison");
}

int sht_debug_withhold_stage(sht_plan_t p, int stage)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (stage < -1) return fail(SHT_EINVAL, "stage < -1");
    std::lock_guard<std::mutex> lk(p->mu);
    p->tc.withhold = stage;
    return SHT_OK;
}

int sht_set_tiles(sht_plan_t p, const int *vals, int n)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (!vals || n < 0 || n > 6) return fail(SHT_EINVAL, "need 0 <= n <= 6 values");
    auto in = [](int v, std::initializer_list<int> ok) {
        for (int o : ok)
            if (v == o) return true;
        return false;
    };
    const bool valid = (n < 1 || in(vals[0], {1, 2, 4})) && (n < 2 || in(vals[1], {1, 2})) &&
                       (n < 3 || in(vals[2], {256, 512})) && (n < 4 || in(vals[3], {1, 2, 4, 8})) &&
                       (n < 5 || in(vals[4], {1, 2, 4, 8, 16})) && (n < 6 || in(vals[5], {1, 2, 4, 8}));
    if (!valid) return fail(SHT_EINVAL, "tile shape outside the candidate set");
    std::lock_guard<std::mutex> lk(p->mu);
    int *dst[6] = {&p->ring_g[0], &p->ring_g[1], &p->ring_nt, &p->fp64_bc, &p->fp64_ring_g, &p->adj_ring_g};
    for (int i = 0; i < n; ++i) *dst[i] = vals[i];
    return SHT_OK;
}

int sht_plan_destroy(sht_plan_t plan)
{
    free_plan(plan);
    return SHT_OK;
}

size_t sht_nalm(sht_plan_t p) { return p ? (size_t)p->nalm : 0; }
size_t sht_npix(sht_plan_t p) { return p ? (size_t)p->npix : 0; }
int sht_nrings(sht_plan_t p) { return p ? p->nrings : 0; }
int sht_lmax(sht_plan_t p) { return p ? p->lmax : 0; }
int sht_mmax(sht_plan_t p) { return p ? p->mmax : 0; }

int sht_alm2map_batch(sht_plan_t p, int nbatch, const void *alm_dev, void *map_dev, int prec,
                      void *stream)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (nbatch < 0) return fail(SHT_EINVAL, "nbatch < 0");
    if (prec != SHT_FP64 && prec != SHT_FP32_TC && prec != SHT_BF16X3_TC && prec != SHT_BF16X6_TC)
        return fail(SHT_EINVAL, "unknown precision %d", prec);
    if (nbatch == 0) return SHT_OK;
    if (!alm_dev || !map_dev) return fail(SHT_EINVAL, "null device pointer");
    if (prec != SHT_FP64) return alm2map_tc(p, nbatch, alm_dev, map_dev, prec, stream);
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard dg(p->device);
    return alm2map_fp64(p, nbatch, static_cast<const double2 *>(alm_dev), static_cast<double *>(map_dev),
                        static_cast<cudaStream_t>(stream));
}

int sht_alm2map(sht_plan_t p, const void *alm_dev, void *map_dev, int prec, void *stream)
{
    return sht_alm2map_batch(p, 1, alm_dev, map_dev, prec, stream);
}

int sht_alm2map_spin2(sht_plan_t p, int nbatch, const void *elm_dev, const void *blm_dev, void *map_dev, int prec,
                      void *stream)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (nbatch < 0) return fail(SHT_EINVAL, "nbatch < 0");
    if (prec != SHT_FP64 && prec != SHT_FP32_TC && prec != SHT_BF16X3_TC && prec != SHT_BF16X6_TC)
        return fail(SHT_EINVAL, "unknown precision %d", prec);
    if (prec != SHT_FP64) return fail(SHT_EUNSUPPORTED, "the spin-2 transform is built for SHT_FP64");
    if (!(p->min_sin > 0.0)) return fail(SHT_EUNSUPPORTED, "spin-2 transform: a ring lies on a pole (sin theta = 0)");
    if (nbatch == 0) return SHT_OK;
    if (!elm_dev || !blm_dev || !map_dev) return fail(SHT_EINVAL, "null device pointer");
    if (2LL * nbatch > 32768) return fail(SHT_EUNSUPPORTED, "nbatch > 16384");
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard dg(p->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t per_map = (size_t)p->nrings * (p->mmax + 1) * sizeof(double2);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)nbatch, max_ws_bytes() / (2 * per_map)));
    if ((rc = ensure_ws(p, 2 * per_map * chunk))) return rc;
    double2 *delta = static_cast<double2 *>(p->ws);
    for (int b0 = 0; b0 < nbatch; b0 += chunk) {
        const int nb = std::min(chunk, nbatch - b0);
        StageScope s1(p, SHT_STAGE_LEGENDRE, st);
        cudaError_t e = sht::launch_legendre_spin2_fp64(p->dp, static_cast<const double2 *>(elm_dev) + (size_t)b0 * p->nalm,
                                                        static_cast<const double2 *>(blm_dev) + (size_t)b0 * p->nalm,
                                                        delta, nb, st);
        s1.done(e);
        if (e != cudaSuccess) return cuda_fail(e, "legendre_spin2_fp64 launch");
        // Q and U of every map are two real syntheses of the ring step
        StageScope s2(p, SHT_STAGE_RING, st);
        e = sht::launch_ring_synth_fp64(p->dp, delta, static_cast<double *>(map_dev) + (size_t)2 * b0 * p->npix, 2 * nb,
                                        p->fp64_ring_g, st);
        s2.done(e, sht::ring_launches(p->dp));
        if (e != cudaSuccess) return cuda_fail(e, "ring_synth_fp64 launch (spin 2)");
    }
    return SHT_OK;
}

int sht_alm2map_host(sht_plan_t p, int nsteps, int nbatch, const void *const *alm_host, void *const *map_host,
                     int prec, void *stream)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (nsteps < 0 || nbatch < 0) return fail(SHT_EINVAL, "nsteps < 0 or nbatch < 0");
    if (prec != SHT_FP64 && prec != SHT_FP32_TC && prec != SHT_BF16X3_TC && prec != SHT_BF16X6_TC)
        return fail(SHT_EINVAL, "unknown precision %d", prec);
    if (nsteps == 0 || nbatch == 0) return SHT_OK;
    if (!alm_host || !map_host) return fail(SHT_EINVAL, "null pointer array");
    for (int k = 0; k < nsteps; ++k)
        if (!alm_host[k] || !map_host[k]) return fail(SHT_EINVAL, "null host pointer for step %d", k);
    const size_t ab = (size_t)nbatch * p->nalm * 16;
    const size_t mb = (size_t)nbatch * p->npix * (prec == SHT_FP64 ? 8 : 4);
    const size_t ab_al = (ab + 255) & ~(size_t)255, mb_al = (mb + 255) & ~(size_t)255;
    cudaStream_t comp = static_cast<cudaStream_t>(stream);
    {
        std::lock_guard<std::mutex> lk(p->mu);
        DeviceGuard dg(p->device);
        cudaError_t e = cudaSuccess;
        if (!p->hp_up) e = cudaStreamCreateWithFlags(&p->hp_up, cudaStreamNonBlocking);
        if (e == cudaSuccess && !p->hp_down) e = cudaStreamCreateWithFlags(&p->hp_down, cudaStreamNonBlocking);
        for (auto &ev : p->hp_ev)
            if (e == cudaSuccess && !ev) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "host pipeline set-up");
        const size_t need = 2 * (ab_al + mb_al);
        if (p->hp_bytes < need) {
            if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
            if (p->hp_buf) cudaFree(p->hp_buf);
            p->hp_buf = nullptr;
            p->hp_bytes = 0;
            if ((e = cudaMalloc(&p->hp_buf, need)) != cudaSuccess) {
                p->hp_buf = nullptr;
                cudaGetLastError();
                return fail(SHT_ENOMEM, "host pipeline buffers cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
            }
            p->hp_bytes = need;
        }
    }
    char *base = static_cast<char *>(p->hp_buf);
    void *d_alm[2] = {base, base + ab_al};
    void *d_map[2] = {base + 2 * ab_al, base + 2 * ab_al + mb_al};
    // events per buffer parity: uploaded, consumed (input buffer free), done, downloaded (output buffer free)
    cudaEvent_t *up_ev = p->hp_ev, *cons_ev = p->hp_ev + 2, *done_ev = p->hp_ev + 4, *down_ev = p->hp_ev + 6;
    DeviceGuard dg(p->device);
    auto upload = [&](int k) -> cudaError_t {
        const int b = k & 1;
        cudaError_t e = cudaSuccess;
        if (k >= 2) e = cudaStreamWaitEvent(p->hp_up, cons_ev[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_alm[b], alm_host[k], ab, cudaMemcpyHostToDevice, p->hp_up);
        if (e == cudaSuccess) e = cudaEventRecord(up_ev[b], p->hp_up);
        return e;
    };
    cudaError_t e = upload(0);
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
        const int b = k & 1;
        if (k + 1 < nsteps && (e = upload(k + 1)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(comp, up_ev[b], 0)) != cudaSuccess) break;
        if (k >= 2 && (e = cudaStreamWaitEvent(comp, down_ev[b], 0)) != cudaSuccess) break;
        if ((rc = sht_alm2map_batch(p, nbatch, d_alm[b], d_map[b], prec, stream))) return rc;
        if ((e = cudaEventRecord(cons_ev[b], comp)) != cudaSuccess) break;
        if ((e = cudaEventRecord(done_ev[b], comp)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(p->hp_down, done_ev[b], 0)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(map_host[k], d_map[b], mb, cudaMemcpyDeviceToHost, p->hp_down)) != cudaSuccess) break;
        if ((e = cudaEventRecord(down_ev[b], p->hp_down)) != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->hp_down);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->hp_up);
    if (e == cudaSuccess) e = cudaStreamSynchronize(comp);
    if (e != cudaSuccess) return cuda_fail(e, "host pipeline");
    return SHT_OK;
}

int sht_map2alm_adjoint_batch(sht_plan_t p, int nbatch, const void *map_dev, void *alm_dev,
                              int prec, void *stream)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (nbatch < 0) return fail(SHT_EINVAL, "nbatch < 0");
    if (prec != SHT_FP64 && prec != SHT_FP32_TC && prec != SHT_BF16X3_TC && prec != SHT_BF16X6_TC)
        return fail(SHT_EINVAL, "unknown precision %d", prec);
    if (nbatch == 0) return SHT_OK;
    if (!alm_dev || !map_dev) return fail(SHT_EINVAL, "null device pointer");
    if (prec != SHT_FP64) {
        std::lock_guard<std::mutex> lk(p->mu);
        DeviceGuard dg(p->device);
        return analysis_tc(p, nbatch, static_cast<const float *>(map_dev), static_cast<double2 *>(alm_dev), nullptr,
                           2.0, prec, static_cast<cudaStream_t>(stream));
    }
    if (sht::legendre_adj_smem_bytes(p->dp, 4) == 0)
        return fail(SHT_EUNSUPPORTED, "adjoint: %d ring pairs exceed the shared-memory state", p->npairs);
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard dg(p->device);
    return analysis_fp64(p, nbatch, static_cast<const double *>(map_dev), static_cast<double2 *>(alm_dev), nullptr,
                         2.0, static_cast<cudaStream_t>(stream));
}

int sht_map2alm_batch(sht_plan_t p, int nbatch, const void *map_dev, void *alm_dev, int prec, int niter,
                      void *stream)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (nbatch < 0 || niter < 0) return fail(SHT_EINVAL, "nbatch < 0 or niter < 0");
    if (prec != SHT_FP64 && prec != SHT_FP32_TC && prec != SHT_BF16X3_TC && prec != SHT_BF16X6_TC)
        return fail(SHT_EINVAL, "unknown precision %d", prec);
    if (nbatch == 0) return SHT_OK;
    if (!alm_dev || !map_dev) return fail(SHT_EINVAL, "null device pointer");
    if (prec != SHT_FP64 && niter > 0)
        return fail(SHT_EUNSUPPORTED, "map2alm refinement steps (niter > 0) are built for SHT_FP64 only");
    if (prec == SHT_FP64 && sht::legendre_adj_smem_bytes(p->dp, 4) == 0)
        return fail(SHT_EUNSUPPORTED, "map2alm: %d ring pairs exceed the shared-memory state", p->npairs);
    std::lock_guard<std::mutex> lk(p->mu);
    bool any = false;
    for (double w : p->wring_h) any = any || w > 0.0;
    if (!any) return fail(SHT_EUNSUPPORTED, "the grid has no quadrature weights (sht_set_ring_weights)");
    DeviceGuard dg(p->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (prec != SHT_FP64)
        return analysis_tc(p, nbatch, static_cast<const float *>(map_dev), static_cast<double2 *>(alm_dev),
                           p->wring_d, 1.0, prec, st);
    const double *map = static_cast<const double *>(map_dev);
    double2 *alm = static_cast<double2 *>(alm_dev);
    if ((rc = analysis_fp64(p, nbatch, map, alm, p->wring_d, 1.0, st))) return rc;
    if (niter == 0) return SHT_OK;
    // Jacobi refinement: a += map2alm(y - alm2map(a)), niter times
    void *res = nullptr, *da = nullptr;
    const long long npx = (long long)nbatch * p->npix, nal = (long long)nbatch * p->nalm;
    cudaError_t e = cudaMalloc(&res, (size_t)npx * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&da, (size_t)nal * sizeof(double2));
    if (e != cudaSuccess) {
        if (res) cudaFree(res);
        if (da) cudaFree(da);
        cudaGetLastError();
        return fail(SHT_ENOMEM, "map2alm iteration buffers: %s", cudaGetErrorString(e));
    }
    for (int it = 0; it < niter && rc == SHT_OK; ++it) {
        rc = alm2map_fp64(p, nbatch, alm, static_cast<double *>(res), st);
        if (rc) break;
        residual_kernel<<<1184, 256, 0, st>>>(map, static_cast<double *>(res), npx);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            rc = cuda_fail(e, "residual launch");
            break;
        }
        g_launches.fetch_add(1, std::memory_order_relaxed);
        rc = analysis_fp64(p, nbatch, static_cast<const double *>(res), static_cast<double2 *>(da), p->wring_d, 1.0,
                           st);
        if (rc) break;
        accumulate_kernel<<<1184, 256, 0, st>>>(alm, static_cast<const double2 *>(da), nal);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            rc = cuda_fail(e, "accumulate launch");
            break;
        }
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    // the buffers may still be in use by the launches just queued on st
    const cudaError_t se = cudaStreamSynchronize(st);
    cudaFree(res);
    cudaFree(da);
    if (rc == SHT_OK && se != cudaSuccess) rc = cuda_fail(se, "cudaStreamSynchronize");
    return rc;
}

int sht_map2alm(sht_plan_t p, const void *map_dev, void *alm_dev, int prec, int niter, void *stream)
{
    return sht_map2alm_batch(p, 1, map_dev, alm_dev, prec, niter, stream);
}

int sht_set_ring_weights(sht_plan_t p, const double *w)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (!w) return fail(SHT_EINVAL, "null weights");
    for (int r = 0; r < p->nrings; ++r)
        if (!(std::isfinite(w[r]) && w[r] >= 0.0)) return fail(SHT_EINVAL, "weight %d not finite and >= 0", r);
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard dg(p->device);
    cudaError_t e = cudaDeviceSynchronize();  // no launch may still read the old weights
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    e = cudaMemcpy(p->wring_d, w, (size_t)p->nrings * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(weights)");
    p->wring_h.assign(w, w + p->nrings);
    return SHT_OK;
}

int sht_ring_weights(sht_plan_t p, double *w)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (!w) return fail(SHT_EINVAL, "null output");
    std::copy(p->wring_h.begin(), p->wring_h.end(), w);
    return SHT_OK;
}

unsigned long long sht_kernel_launches(void) { return g_launches.load(); }

int sht_sync(sht_plan_t p)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    DeviceGuard dg(p->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    int st = 0;
    e = cudaMemcpy(&st, p->tc.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (st != 0) {
        const int zero = 0;
        cudaMemcpy(p->tc.status, &zero, sizeof(int), cudaMemcpyHostToDevice);
        return fail(SHT_ETIMEOUT, "a bounded device-side wait gave up (kernel status %d)", st);
    }
    return SHT_OK;
}

int sht_profile(sht_plan_t p, int enable)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(p->mu);
    p->profiling = enable != 0;
    return SHT_OK;
}

int sht_profile_read(sht_plan_t p, int nstage, double *ms, long long *launches)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (nstage < 0) return fail(SHT_EINVAL, "nstage < 0");
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard dg(p->device);
    for (auto &e : p->prof_pending) {
        cudaError_t err = cudaEventSynchronize(e.b);
        float t = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e.a, e.b);
        if (err != cudaSuccess) return cuda_fail(err, "profiling event");
        p->prof_ms[e.stage] += t;
        p->prof_n[e.stage] += 1;
        p->prof_pool.push_back(e.a);
        p->prof_pool.push_back(e.b);
    }
    p->prof_pending.clear();
    for (int i = 0; i < nstage; ++i) {
        if (ms) ms[i] = i < SHT_NSTAGES ? p->prof_ms[i] : 0.0;
        if (launches) launches[i] = i < SHT_NSTAGES ? p->prof_n[i] : 0;
    }
    for (int i = 0; i < SHT_NSTAGES; ++i) {
        p->prof_ms[i] = 0.0;
        p->prof_n[i] = 0;
    }
    return SHT_OK;
}

int sht_map2alm_adjoint(sht_plan_t p, const void *map_dev, void *alm_dev, int prec, void *stream)
{
    return sht_map2alm_adjoint_batch(p, 1, map_dev, alm_dev, prec, stream);
}

}  // extern "C"

// ------------------------------------------------ partitioned transform --
// Algorithm 3 of the paper: the orders m are split over parts for the
// Legendre step, Delta is exchanged all-to-all, and the rings are split over
// parts for the ring step.  The library computes each part's share; the
// exchange between parts (GPUs) is the caller's (e.g. an NCCL all-to-all).

namespace {

struct PartLayout {
    std::vector<int> mlist;             // this part's orders, ascending
    std::vector<std::vector<int>> rings;  // rings of every part, ascending
    std::vector<std::vector<int>> ms;     // orders of every part, ascending
};

int part_layout(const sht_plan_s *p, int nparts, const int *m_owner, const int *ring_owner, int part, PartLayout &pl)
{
    if (nparts < 1 || part < 0 || part >= nparts) return fail(SHT_EINVAL, "need 0 <= part < nparts");
    if (!m_owner || !ring_owner) return fail(SHT_EINVAL, "null owner array");
    pl.rings.assign(nparts, {});
    pl.ms.assign(nparts, {});
    for (int m = 0; m <= p->mmax; ++m) {
        if (m_owner[m] < 0 || m_owner[m] >= nparts) return fail(SHT_EINVAL, "m_owner[%d] = %d outside [0, %d)", m, m_owner[m], nparts);
        pl.ms[m_owner[m]].push_back(m);
    }
    for (int r = 0; r < p->nrings; ++r) {
        if (ring_owner[r] < 0 || ring_owner[r] >= nparts)
            return fail(SHT_EINVAL, "ring_owner[%d] = %d outside [0, %d)", r, ring_owner[r], nparts);
        pl.rings[ring_owner[r]].push_back(r);
    }
    pl.mlist = pl.ms[part];
    return SHT_OK;
}

// Device copy of host tables into the plan's partition scratch (synchronous:
// waits for the work already queued on st, which may still read the tables).
int part_upload(sht_plan_s *p, const std::vector<std::pair<const void *, size_t>> &parts, std::vector<char *> &out,
                cudaStream_t st)
{
    cudaError_t e0 = cudaStreamSynchronize(st);
    if (e0 != cudaSuccess) return cuda_fail(e0, "cudaStreamSynchronize");
    size_t need = 0;
    for (auto &q : parts) need += (q.second + 255) & ~(size_t)255;
    if (p->part_bytes < need) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
        if (p->part_buf) cudaFree(p->part_buf);
        p->part_buf = nullptr;
        p->part_bytes = 0;
        if ((e = cudaMalloc(&p->part_buf, need)) != cudaSuccess) {
            p->part_buf = nullptr;
            cudaGetLastError();
            return fail(SHT_ENOMEM, "partition tables cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
        }
        p->part_bytes = need;
    }
    char *b = static_cast<char *>(p->part_buf);
    out.clear();
    for (auto &q : parts) {
        if (q.second) {
            cudaError_t e = cudaMemcpy(b, q.first, q.second, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "partition tables");
        }
        out.push_back(b);
        b += (q.second + 255) & ~(size_t)255;
    }
    return SHT_OK;
}

}  // namespace

extern "C" int sht_partition(int lmax, int mmax, int nrings, const int *nphi, int nparts, int *m_owner,
                             int *ring_owner)
{
    g_err.clear();
    if (lmax < 0 || mmax < 0 || mmax > lmax || nrings < 1 || nparts < 1 || !nphi || !m_owner || !ring_owner)
        return fail(SHT_EINVAL, "sht_partition: bad arguments");
    const int L = lmax, M = mmax;
    // orders in pairs (m, M - m), whose recurrence lengths (L - m + 1) sum to a
    // constant when L = M, each pair (longest first) to the part with the least
    // work so far
    std::vector<std::pair<long long, std::pair<int, int>>> units;
    for (int m = 0; 2 * m <= M; ++m) {
        const int m2 = M - m;
        const long long c = (L - m + 1) + (m2 != m ? (L - m2 + 1) : 0);
        units.push_back({c, {m, m2}});
    }
    std::stable_sort(units.begin(), units.end(),
                     [](const std::pair<long long, std::pair<int, int>> &a,
                        const std::pair<long long, std::pair<int, int>> &b) { return a.first > b.first; });
    std::vector<long long> load(nparts, 0);
    for (auto &u : units) {
        const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[q] += u.first;
        m_owner[u.second.first] = q;
        m_owner[u.second.second] = q;
    }
    // rings in contiguous ranges of about equal pixel count: ring r goes to the
    // part whose share [q total / nparts, (q + 1) total / nparts) holds its first pixel
    long long total = 0;
    for (int r = 0; r < nrings; ++r) {
        if (nphi[r] < 1) return fail(SHT_EINVAL, "sht_partition: nphi[%d] < 1", r);
        total += nphi[r];
    }
    long long first = 0;
    int q = 0;
    for (int r = 0; r < nrings; ++r) {
        while (q + 1 < nparts && first >= (total * (q + 1)) / nparts) ++q;
        ring_owner[r] = q;
        first += nphi[r];
    }
    return SHT_OK;
}

extern "C" int sht_ring_lengths(sht_plan_t p, int *nphi)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (!nphi) return fail(SHT_EINVAL, "null output array");
    std::copy(p->nphi_h.begin(), p->nphi_h.end(), nphi);
    return SHT_OK;
}

extern "C" int sht_alm2map_mpart(sht_plan_t p, int nbatch, int nparts, const int *m_owner, const int *ring_owner,
                                 int part, const void *alm_dev, void *send_dev, int prec, void *stream)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (nbatch < 0) return fail(SHT_EINVAL, "nbatch < 0");
    if (prec != SHT_FP64) return fail(SHT_EUNSUPPORTED, "the partitioned transform is built for SHT_FP64");
    PartLayout pl;
    if ((rc = part_layout(p, nparts, m_owner, ring_owner, part, pl))) return rc;
    if (nbatch == 0 || pl.mlist.empty()) return SHT_OK;
    if (!alm_dev || !send_dev) return fail(SHT_EINVAL, "null device pointer");
    const int nm = (int)pl.mlist.size();
    // send layout: for destination q, its rings' rows [row][map][order of this part]
    std::vector<long long> row_off(p->nrings);
    long long off = 0;
    for (int q = 0; q < nparts; ++q)
        for (size_t i = 0; i < pl.rings[q].size(); ++i) {
            row_off[pl.rings[q][i]] = off;
            off += (long long)nbatch * nm;
        }
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard dg(p->device);
    std::vector<char *> d;
    if ((rc = part_upload(p, {{pl.mlist.data(), pl.mlist.size() * sizeof(int)},
                              {row_off.data(), row_off.size() * sizeof(long long)}},
                          d, static_cast<cudaStream_t>(stream))))
        return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    StageScope s1(p, SHT_STAGE_LEGENDRE, st);
    cudaError_t e = sht::launch_legendre_mpart_fp64(p->dp, static_cast<const double2 *>(alm_dev),
                                                    static_cast<double2 *>(send_dev), nbatch,
                                                    reinterpret_cast<const int *>(d[0]), nm,
                                                    reinterpret_cast<const long long *>(d[1]), st);
    s1.done(e);
    if (e != cudaSuccess) return cuda_fail(e, "legendre_mpart launch");
    return SHT_OK;
}

extern "C" int sht_ring_synth_part(sht_plan_t p, int nbatch, int nparts, const int *m_owner, const int *ring_owner,
                                   int part, const void *recv_dev, void *map_dev, int prec, void *stream)
{
    g_err.clear();
    int rc = check_plan(p);
    if (rc) return rc;
    if (nbatch < 0) return fail(SHT_EINVAL, "nbatch < 0");
    if (prec != SHT_FP64) return fail(SHT_EUNSUPPORTED, "the partitioned transform is built for SHT_FP64");
    PartLayout pl;
    if ((rc = part_layout(p, nparts, m_owner, ring_owner, part, pl))) return rc;
    const std::vector<int> &mine = pl.rings[part];
    if (nbatch == 0 || mine.empty()) return SHT_OK;
    if (!recv_dev || !map_dev) return fail(SHT_EINVAL, "null device pointer");
    const int nrows = (int)mine.size();
    if (nbatch > 32768) return fail(SHT_EUNSUPPORTED, "nbatch > 32768");
    // receive layout: block of source q = [row][map][order of q]
    std::vector<long long> m_off(p->mmax + 1);
    std::vector<int> m_cnt(p->mmax + 1), m_col(p->mmax + 1);
    long long off = 0;
    for (int q = 0; q < nparts; ++q) {
        for (size_t i = 0; i < pl.ms[q].size(); ++i) {
            const int m = pl.ms[q][i];
            m_off[m] = off;
            m_cnt[m] = (int)pl.ms[q].size();
            m_col[m] = (int)i;
        }
        off += (long long)nrows * nbatch * (long long)pl.ms[q].size();
    }
    std::vector<int> row(p->nrings, -1), rs, rb;
    for (int i = 0; i < nrows; ++i) row[mine[i]] = i;
    for (int r : p->rings_smooth_h)
        if (row[r] >= 0) rs.push_back(r);
    for (int r : p->rings_blue_h)
        if (row[r] >= 0) rb.push_back(r);
    std::lock_guard<std::mutex> lk(p->mu);
    DeviceGuard dg(p->device);
    const size_t dbytes = (size_t)nbatch * nrows * (p->mmax + 1) * sizeof(double2);
    if ((rc = ensure_ws(p, dbytes))) return rc;
    std::vector<char *> d;
    if ((rc = part_upload(p, {{m_off.data(), m_off.size() * sizeof(long long)},
                              {m_cnt.data(), m_cnt.size() * sizeof(int)},
                              {m_col.data(), m_col.size() * sizeof(int)},
                              {row.data(), row.size() * sizeof(int)},
                              {rs.data(), rs.size() * sizeof(int)},
                              {rb.data(), rb.size() * sizeof(int)}},
                          d, static_cast<cudaStream_t>(stream))))
        return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double2 *delta = static_cast<double2 *>(p->ws);
    cudaError_t e = sht::launch_delta_gather(static_cast<const double2 *>(recv_dev), delta, nbatch, nrows, p->mmax,
                                             reinterpret_cast<const long long *>(d[0]),
                                             reinterpret_cast<const int *>(d[1]),
                                             reinterpret_cast<const int *>(d[2]), st);
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    if (e != cudaSuccess) return cuda_fail(e, "delta gather launch");
    DevPlan q = p->dp;
    q.ring_row = reinterpret_cast<const int *>(d[3]);
    q.delta_rows = nrows;
    q.rings_smooth = rs.empty() ? nullptr : reinterpret_cast<const int *>(d[4]);
    q.n_smooth = (int)rs.size();
    q.rings_blue = rb.empty() ? nullptr : reinterpret_cast<const int *>(d[5]);
    q.n_blue = (int)rb.size();
    StageScope s2(p, SHT_STAGE_RING, st);
    e = sht::launch_ring_synth_fp64(q, delta, static_cast<double *>(map_dev), nbatch, p->fp64_ring_g, st);
    s2.done(e, sht::ring_launches(q));
    if (e != cudaSuccess) return cuda_fail(e, "ring_synth_part launch");
    return SHT_OK;
}

// ----------------------------------------------------------- multi-request --

struct sht_multi_s {
    int nreq = 0, prec = 0, device = 0, nctas = 0;
    int nsm = 1;         // SMs of the device
    int ring_nt = 256;   // tensor-core forms: threads per CTA of the shared-memory ring kernel
    std::vector<sht_plan_t> plans;
    std::vector<size_t> delta_ofs;  // bytes, per request
    std::vector<void *> allocs;
    sht::DevPlan *d_plans = nullptr;
    int4 *d_items = nullptr;
    int *d_cta_off = nullptr;  // tensor-core forms: CTA ranges of d_items
    int nitems = 0, ctas = 0;
    int2 *d_smooth = nullptr, *d_blue = nullptr;
    int n_smooth = 0, n_blue = 0, smooth_cap = 0, blue_cap = 0;
    // tensor-core forms: (request, ring) units of the register-FFT ring kernel
    int2 *d_rf = nullptr;
    int n_rf = 0, rf_mmax = 0;
    // tensor-core forms: (request, m) items of the one-launch operand prep
    int2 *d_prep = nullptr;
    int n_prep = 0;
    int *d_counter = nullptr;
    void *d_delta = nullptr;
    // tensor-core forms: a request whose plan already appeared earlier in the
    // list gets its own B-operand buffer (nullptr: the plan's own)
    std::vector<void *> bbuf_own;
};

namespace {

void free_multi(sht_multi_s *q)
{
    if (!q) return;
    {
        DeviceGuard g(q->device);
        cudaDeviceSynchronize();
        for (void *d : q->allocs) cudaFree(d);
    }
    delete q;
}

template <typename T>
int multi_upload(sht_multi_s *q, const std::vector<T> &h, T **out)
{
    *out = nullptr;
    if (h.empty()) return SHT_OK;
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, h.size() * sizeof(T));
    if (e != cudaSuccess) return fail(SHT_ENOMEM, "cudaMalloc(%zu): %s", h.size() * sizeof(T), cudaGetErrorString(e));
    q->allocs.push_back(d);
    e = cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    *out = static_cast<T *>(d);
    return SHT_OK;
}

}  // namespace

extern "C" int sht_multi_create(int nreq, const sht_plan_t *plans, int prec, sht_multi_t *out)
{
    g_err.clear();
    if (!out) return fail(SHT_EINVAL, "null output pointer");
    *out = nullptr;
    if (nreq < 1 || nreq > sht::kMaxReq) return fail(SHT_EINVAL, "need 1 <= nreq <= %d", sht::kMaxReq);
    if (!plans) return fail(SHT_EINVAL, "null plan array");
    if (prec != SHT_FP64 && prec != SHT_FP32_TC && prec != SHT_BF16X3_TC && prec != SHT_BF16X6_TC)
        return fail(SHT_EINVAL, "unknown precision %d", prec);
    for (int i = 0; i < nreq; ++i) {
        if (!plans[i]) return fail(SHT_EINVAL, "null plan %d", i);
        if (plans[i]->device != plans[0]->device) return fail(SHT_EINVAL, "plans on different devices");
    }
    auto *q = new (std::nothrow) sht_multi_s();
    if (!q) return fail(SHT_ENOMEM, "multi allocation");
    q->nreq = nreq;
    q->prec = prec;
    q->device = plans[0]->device;
    q->plans.assign(plans, plans + nreq);
    DeviceGuard dg(q->device);
    int rc = SHT_OK;
    if (prec == SHT_FP64) {
        // work list (request, m, ring block) by decreasing cost, ring items, Delta offsets
        struct Item {
            long long cost;
            int4 w;
        };
        std::vector<Item> items;
        std::vector<int2> smooth, blue;
        std::vector<sht::DevPlan> dp(nreq);
        size_t dofs = 0;
        for (int i = 0; i < nreq; ++i) {
            const sht_plan_s *p = plans[i];
            dp[i] = p->dp;
            const int nrb = (p->npairs + 127) / 128;
            std::vector<int> g0((size_t)nrb * (p->mmax + 1), 0);
            if (p->dp.skip_g) {
                cudaError_t e = cudaMemcpy(g0.data(), p->dp.skip_g, g0.size() * sizeof(int), cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "skip tables");
                    break;
                }
            }
            // cost: the degrees the item's recurrence runs plus a fixed share
            // for its setup and Delta epilogue
            for (int m = 0; m <= p->mmax; ++m)
                for (int rb = 0; rb < nrb; ++rb)
                    items.push_back({(long long)(p->lmax - m + 1) - 64LL * g0[(size_t)m * nrb + rb] + kItemOverhead,
                                     make_int4(i, m, rb, 0)});
            for (int r : p->rings_smooth_h) smooth.push_back(make_int2(i, r));
            for (int r : p->rings_blue_h) blue.push_back(make_int2(i, r));
            q->smooth_cap = std::max(q->smooth_cap, p->dp.fft_cap);
            q->blue_cap = std::max(q->blue_cap, p->dp.blue_cap);
            q->delta_ofs.push_back(dofs);
            dofs += (size_t)p->nrings * (p->mmax + 1) * sizeof(double2);
            dofs = (dofs + 255) & ~(size_t)255;
        }
        // longest first to the CTA with the least work so far, stored CTA-major
        std::stable_sort(items.begin(), items.end(), [](const Item &a, const Item &b) { return a.cost > b.cost; });
        int nsm_tc = 0;
        cudaDeviceGetAttribute(&nsm_tc, cudaDevAttrMultiProcessorCount, q->device);
        const int n = (int)items.size();
        const int G = std::max(1, std::min(n, nsm_tc));
        std::vector<long long> cost((size_t)n);
        for (int j = 0; j < n; ++j) cost[j] = items[j].cost;
        std::vector<int> coff((size_t)G + 1), order((size_t)n);
        build_work_lists(n, cost.data(), G, coff.data(), order.data());
        std::vector<int4> w((size_t)n);
        for (int j = 0; j < n; ++j) w[j] = items[order[j]].w;
        q->ctas = G;
        q->nitems = (int)w.size();
        q->n_smooth = (int)smooth.size();
        q->n_blue = (int)blue.size();
        if ((rc = multi_upload(q, dp, &q->d_plans)) || (rc = multi_upload(q, w, &q->d_items)) ||
            (rc = multi_upload(q, coff, &q->d_cta_off)) ||
            (rc = multi_upload(q, smooth, &q->d_smooth)) || (rc = multi_upload(q, blue, &q->d_blue))) {
            std::string keep = g_err;
            free_multi(q);
            g_err = keep;
            return rc;
        }
        cudaError_t e = cudaMalloc(&q->d_counter, sizeof(int));
        if (e == cudaSuccess) {
            q->allocs.push_back(q->d_counter);
            e = cudaMalloc(&q->d_delta, dofs);
            if (e == cudaSuccess) q->allocs.push_back(q->d_delta);
        }
        if (e != cudaSuccess) {
            free_multi(q);
            return fail(SHT_ENOMEM, "multi workspace: %s", cudaGetErrorString(e));
        }
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, q->device);
        q->nctas = std::max(1, nsm) * 8;  // persistent CTAs: several per SM hide the FP64 latency
        q->nsm = std::max(1, nsm);
    } else {
        // tensor-core forms: each plan's B operand buffer and skip tables, then
        // one work list (request, m, ring block) by decreasing cost for one
        // persistent Legendre launch, merged ring lists, Delta [ring][m] per request
        struct Item {
            long long cost;
            int4 w;
        };
        std::vector<Item> items;
        std::vector<int2> smooth, blue;
        std::vector<std::pair<double, int2>> rf;
        std::vector<int2> prep;
        std::vector<sht::DevPlan> dp(nreq);
        size_t dofs = 0;
        q->bbuf_own.assign(nreq, nullptr);
        for (int i = 0; i < nreq; ++i) {
            sht_plan_s *p = plans[i];
            std::lock_guard<std::mutex> lk(p->mu);
            if ((rc = ensure_tc(p, prec)) || (rc = ensure_warm(p, nullptr))) break;
            if (std::find(plans, plans + i, p) != plans + i) {
                // the plan serves an earlier request too: its operand buffer is taken
                void *b = nullptr;
                cudaError_t e = cudaMalloc(&b, sht::tc_bbuf_bytes(p->tc, prec));
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    rc = fail(SHT_ENOMEM, "operand buffer of repeated plan %d: %s", i, cudaGetErrorString(e));
                    break;
                }
                q->allocs.push_back(b);
                q->bbuf_own[i] = b;
            }
            dp[i] = p->dp;
            const int nrb = (p->npairs + 127) / 128;
            // items past every ring of their block (Delta exactly zero there) are left out
            const bool cut = p->dp.ring_mlim && (int)p->blim_h.size() == nrb;
            for (int m = 0; m <= p->mmax; ++m)
                for (int rb = 0; rb < nrb; ++rb) {
                    if (cut && m >= p->blim_h[rb]) continue;
                    const long long rows = std::min(128, p->npairs - rb * 128);
                    items.push_back({(long long)(p->lmax - m + 1) * rows, make_int4(i, m, rb, 0)});
                }
            for (int m = 0; m <= p->mmax; ++m) prep.push_back(make_int2(i, m));
            const auto &fs = p->rf_set[p->rf_mode];
            for (int r : fs.rest_s_h) smooth.push_back(make_int2(i, r));
            for (int r : fs.rest_b_h) blue.push_back(make_int2(i, r));
            for (int r : fs.rings_h) rf.push_back({rf_unit_cost(p, r), make_int2(i, r)});
            if (!fs.rings_h.empty()) q->rf_mmax = std::max(q->rf_mmax, p->mmax);
            q->smooth_cap = std::max(q->smooth_cap, p->dp.fft_cap);
            q->blue_cap = std::max(q->blue_cap, p->dp.blue_cap);
            q->delta_ofs.push_back(dofs);
            dofs += (size_t)p->nrings * (p->mmax + 1) * sizeof(float2);
            dofs = (dofs + 255) & ~(size_t)255;
        }
        if (rc) {
            std::string keep = g_err;
            free_multi(q);
            g_err = keep;
            return rc;
        }
        std::stable_sort(items.begin(), items.end(), [](const Item &a, const Item &b) { return a.cost > b.cost; });
        std::vector<int4> w(items.size());
        for (size_t j = 0; j < items.size(); ++j) w[j] = items[j].w;
        q->nitems = (int)w.size();
        q->n_smooth = (int)smooth.size();
        q->n_blue = (int)blue.size();
        std::stable_sort(rf.begin(), rf.end(),
                         [](const std::pair<double, int2> &a, const std::pair<double, int2> &b) { return a.first > b.first; });
        std::vector<int2> rfu(rf.size());
        for (size_t j = 0; j < rf.size(); ++j) rfu[j] = rf[j].second;
        q->n_rf = (int)rfu.size();
        q->n_prep = (int)prep.size();
        if ((rc = multi_upload(q, dp, &q->d_plans)) || (rc = multi_upload(q, w, &q->d_items)) ||
            (rc = multi_upload(q, smooth, &q->d_smooth)) || (rc = multi_upload(q, blue, &q->d_blue)) ||
            (rc = multi_upload(q, rfu, &q->d_rf)) || (rc = multi_upload(q, prep, &q->d_prep))) {
            std::string keep = g_err;
            free_multi(q);
            g_err = keep;
            return rc;
        }
        cudaError_t e = cudaMalloc(&q->d_delta, dofs);
        if (e != cudaSuccess) {
            free_multi(q);
            return fail(SHT_ENOMEM, "multi workspace: %s", cudaGetErrorString(e));
        }
        q->allocs.push_back(q->d_delta);
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, q->device);
        q->nsm = std::max(1, nsm);
        q->nctas = 8 * q->nsm;  // the FP64 launch's setting, kept for sht_multi_tiles
    }
    *out = q;
    return SHT_OK;
}

extern "C" int sht_multi_destroy(sht_multi_t q)
{
    free_multi(q);
    return SHT_OK;
}

extern "C" int sht_multi_debug_poison_delta(sht_multi_t q)
{
    g_err.clear();
    if (!q) return fail(SHT_EINVAL, "null multi context");
    DeviceGuard dg(q->device);
    size_t bytes = 0;
    if (!q->d_delta) return SHT_OK;
    for (int i = 0; i < (int)q->plans.size(); ++i) {
        const sht_plan_s *p = q->plans[i];
        const size_t el = q->prec == SHT_FP64 ? sizeof(double2) : sizeof(float2);
        bytes = std::max(bytes, q->delta_ofs[i] + (size_t)p->nrings * (p->mmax + 1) * el);
    }
    cudaError_t e = cudaMemset(q->d_delta, 0xFF, bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? SHT_OK : cuda_fail(e, "poison");
}

extern "C" int sht_multi_alm2map(sht_multi_t q, const void *const *alm_dev, void *const *map_dev, void *stream)
{
    g_err.clear();
    if (!q) return fail(SHT_EINVAL, "null multi handle");
    if (!alm_dev || !map_dev) return fail(SHT_EINVAL, "null pointer array");
    for (int i = 0; i < q->nreq; ++i)
        if (!alm_dev[i] || !map_dev[i]) return fail(SHT_EINVAL, "null device pointer for request %d", i);
    if (q->prec != SHT_FP64) {
        // tensor-core forms: the operand prep of every request, one persistent
        // Legendre launch over all requests' work items, one ring launch per list
        DeviceGuard dg(q->device);
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const bool bf16 = q->prec != SHT_FP32_TC;
        sht::MultiTcPtrs mp{};
        for (int i = 0; i < q->nreq; ++i) {
            const sht_plan_s *p = q->plans[i];
            mp.alm[i] = alm_dev[i];
            mp.bbuf[i] = q->bbuf_own[i] ? q->bbuf_own[i] : p->tc.bbuf;
            mp.seg[i] = bf16 ? p->tc.seg_bf16 : p->tc.seg_tf32;
            mp.delta[i] = static_cast<char *>(q->d_delta) + q->delta_ofs[i];
            mp.map[i] = map_dev[i];
            mp.cta_off = q->d_cta_off;
            mp.ctas = q->ctas;
        }
        cudaError_t e = sht::launch_tc_prep_multi(q->d_plans, q->d_prep, q->n_prep, mp, q->prec, st);
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core operand prep launch");
        g_launches.fetch_add(1, std::memory_order_relaxed);
        e = sht::launch_tc_main_multi(q->plans[0]->dp, q->d_plans, q->d_items, q->nitems, mp, q->prec,
                                                  q->plans[0]->tc.status, st);
        if (e != cudaSuccess) return cuda_fail(e, "legendre_tc multi launch");
        g_launches.fetch_add(1, std::memory_order_relaxed);
        e = sht::launch_ring_reg_multi(q->plans[0]->dp, q->d_plans, q->d_rf, q->n_rf, q->rf_mmax, mp,
                                       q->plans[0]->tc.status, st);
        if (e != cudaSuccess) return cuda_fail(e, "ring_reg multi launch");
        g_launches.fetch_add(q->n_rf > 0, std::memory_order_relaxed);
        e = sht::launch_ring_synth_mf_multi(q->d_plans, q->d_smooth, q->n_smooth, q->smooth_cap, q->d_blue, q->n_blue,
                                            q->blue_cap, mp, q->ring_nt, st);
        if (e != cudaSuccess) return cuda_fail(e, "ring_synth_mf multi launch");
        g_launches.fetch_add((q->n_smooth > 0) + (q->n_blue > 0), std::memory_order_relaxed);
        return SHT_OK;
    }
    DeviceGuard dg(q->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    sht::MultiPtrs ptrs{};
    for (int i = 0; i < q->nreq; ++i) {
        ptrs.alm[i] = alm_dev[i];
        ptrs.map[i] = map_dev[i];
        ptrs.delta[i] = static_cast<char *>(q->d_delta) + q->delta_ofs[i];
    }
    cudaError_t e = cudaMemsetAsync(q->d_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    e = sht::launch_legendre_multi_fp64(q->d_plans, q->d_items, q->nitems, q->d_counter, ptrs, q->nctas, st);
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    else return cuda_fail(e, "legendre_multi_fp64 launch");
    e = sht::launch_ring_synth_multi_fp64(q->d_plans, q->d_smooth, q->n_smooth, q->smooth_cap, q->d_blue, q->n_blue,
                                          q->blue_cap, ptrs, st);
    if (e != cudaSuccess) return cuda_fail(e, "ring_synth_multi launch");
    g_launches.fetch_add((q->n_smooth > 0) + (q->n_blue > 0), std::memory_order_relaxed);
    return SHT_OK;
}

// Tile shapes of a multi-request context: vals[0] = persistent CTAs per SM of
// the FP64 Legendre launch, vals[1] = threads per CTA of the tensor-core
// forms' shared-memory ring kernel.  Results do not depend on them.
extern "C" int sht_multi_tiles(sht_multi_t q, int *out, int n)
{
    g_err.clear();
    if (!q || !out || n < 2) return fail(SHT_EINVAL, "null multi handle or array, or n < 2");
    out[0] = q->nctas / q->nsm;
    out[1] = q->ring_nt;
    return SHT_OK;
}

extern "C" int sht_multi_set_tiles(sht_multi_t q, const int *vals, int n)
{
    g_err.clear();
    if (!q || !vals || n < 2) return fail(SHT_EINVAL, "null multi handle or array, or n < 2");
    if (vals[0] < 1 || vals[0] > 32) return fail(SHT_EINVAL, "CTAs per SM %d not in 1..32", vals[0]);
    if (vals[1] != 256 && vals[1] != 512) return fail(SHT_EINVAL, "ring threads %d not 256 or 512", vals[1]);
    q->nctas = vals[0] * q->nsm;
    q->ring_nt = vals[1];
    return SHT_OK;
}

// Times every candidate tile shape of the context on the caller's requests
// (one untimed call, then one call timed with events on `stream`) and keeps
// the fastest; the maps are overwritten by the last call.
extern "C" int sht_multi_autotune(sht_multi_t q, const void *const *alm_dev, void *const *map_dev, void *stream)
{
    g_err.clear();
    if (!q) return fail(SHT_EINVAL, "null multi handle");
    DeviceGuard dg(q->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<std::pair<int, int>> cand;
    if (q->prec == SHT_FP64) {
        for (int c : {2, 4, 8, 16}) cand.push_back({c, q->ring_nt});
    } else {
        for (int t : {256, 512}) cand.push_back({q->nctas / q->nsm, t});
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    int rc = SHT_OK;
    float best = 1e30f;
    std::pair<int, int> pick = cand[0];
    for (const auto &c : cand) {
        const int v[2] = {c.first, c.second};
        if ((rc = sht_multi_set_tiles(q, v, 2)) || (rc = sht_multi_alm2map(q, alm_dev, map_dev, stream))) break;
        cudaEventRecord(e0, st);
        if ((rc = sht_multi_alm2map(q, alm_dev, map_dev, stream))) break;
        cudaEventRecord(e1, st);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
            rc = cuda_fail(e, "autotune timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            pick = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int v[2] = {pick.first, pick.second};
    sht_multi_set_tiles(q, v, 2);
    return rc;
}

extern "C" int sht_alm2map_multi(int nreq, const sht_plan_t *plans, const void *const *alm_dev,
                                 void *const *map_dev, int prec, void *stream)
{
    sht_multi_t q = nullptr;
    int rc = sht_multi_create(nreq, plans, prec, &q);
    if (rc) return rc;
    rc = sht_multi_alm2map(q, alm_dev, map_dev, stream);
    if (rc == SHT_OK) {
        cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    }
    std::string keep = g_err;
    sht_multi_destroy(q);
    g_err = keep;
    return rc;
}

// Internal hooks for other translation units of the library (not C ABI).
namespace sht {
const DevPlan *plan_dev(sht_plan_t p) { return p ? &p->dp : nullptr; }
void plan_fp64_tiles(sht_plan_t p, int *bc, int *ring_g)
{
    *bc = p ? p->fp64_bc : 0;
    *ring_g = p ? p->fp64_ring_g : 0;
}
int plan_device(sht_plan_t p) { return p ? p->device : -1; }
std::mutex *plan_mutex(sht_plan_t p) { return p ? &p->mu : nullptr; }
int record_error(int code, const char *msg) { return fail(code, "%s", msg); }
int record_cuda_error(cudaError_t e, const char *what) { return cuda_fail(e, what); }
void clear_error() { g_err.clear(); }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace sht
