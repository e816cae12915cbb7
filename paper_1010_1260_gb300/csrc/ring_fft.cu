// Ring step of alm2map (Eq. Delta2map, sec. 2.2.2): for every ring r,
//   s_r(j) = sum_{m=-M..M} Delta_m(r) e^{i m (phi0_r + 2 pi j / n)},  n = n_phi(r),
// with Delta_{-m} = conj(Delta_m).  Steps, all inside one CTA per (ring, map):
//   1. phase shift and fold: F_k = sum_{m = k mod n} Delta_m e^{i m phi0}
//      + sum_{m >= 1, -m = k mod n} conj(Delta_m e^{i m phi0}) for k = 0..n/2
//      (modes beyond the ring's Nyquist frequency alias onto its bins; the
//      paper defers this "wrapping" to Gorski et al. 2005);
//   2. real inverse DFT of length n.  For even n it runs as one complex DFT of
//      length h = n/2: Z_k = (F_k + conj F_{h-k}) + i w^k (F_k - conj F_{h-k}),
//      w = e^{2 pi i / n}, z = IDFT_h(Z), s_{2j} = Re z_j, s_{2j+1} = Im z_j.
//      Odd n runs the full-length complex DFT of the Hermitian spectrum.
//   3. the complex DFT is a self-sorting (Stockham) mixed-radix transform in
//      shared memory, ping-ponging between two buffers: radix 4, 2, 3, 5
//      butterflies, and a direct pass for any other prime factor.
// Twiddles come from per-plan tables T_n[q] = e^{i pi q / n}, q < 2n, one per
// distinct ring length; HEALPix and Gauss-Legendre rings have
// phi0 = pi * ps / n with an integer ps, so e^{i m phi0} = T_n[(m ps) mod 2n].
#include "sht_internal.cuh"

#include <algorithm>

namespace sht {
namespace {

constexpr int kThreads = 256;
constexpr int kRingGroup = 8;  // maps per CTA: the ring's twiddles are built once per group

int ring_group(int nmaps) { return nmaps < kRingGroup ? nmaps : kRingGroup; }

template <typename R> struct C2T;
template <> struct C2T<double> { using type = double2; };
template <> struct C2T<float> { using type = float2; };

template <typename R>
__device__ __forceinline__ typename C2T<R>::type mk(R x, R y)
{
    typename C2T<R>::type c;
    c.x = x;
    c.y = y;
    return c;
}
// Products and fused multiply-adds with explicit rounding: the compiler may
// not contract them differently in different instantiations, so results do
// not depend on the launch shape (maps per CTA, threads per CTA).
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    C c;
    c.x = rfma(a.x, b.x, -rmul(a.y, b.y));
    c.y = rfma(a.x, b.y, rmul(a.y, b.x));
    return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b)
{
    a.x += b.x;
    a.y += b.y;
    return a;
}
template <typename C> __device__ __forceinline__ C csub(C a, C b)
{
    a.x -= b.x;
    a.y -= b.y;
    return a;
}
template <typename C> __device__ __forceinline__ C cconj(C a)
{
    a.y = -a.y;
    return a;
}
// multiply by +i
template <typename C> __device__ __forceinline__ C cmuli(C a)
{
    C c;
    c.x = -a.y;
    c.y = a.x;
    return c;
}

template <typename R> __device__ __forceinline__ const typename C2T<R>::type *tw_table(const DevPlan &P);
template <> __device__ __forceinline__ const double2 *tw_table<double>(const DevPlan &P) { return P.tw64; }
template <> __device__ __forceinline__ const float2 *tw_table<float>(const DevPlan &P) { return P.tw32; }
template <typename R> __device__ __forceinline__ const typename C2T<R>::type *bhat_table(const DevPlan &P);
template <> __device__ __forceinline__ const double2 *bhat_table<double>(const DevPlan &P) { return P.bhat64; }
template <> __device__ __forceinline__ const float2 *bhat_table<float>(const DevPlan &P) { return P.bhat32; }
template <typename R> __device__ __forceinline__ const typename C2T<R>::type *w2_table(const DevPlan &P);
template <> __device__ __forceinline__ const double2 *w2_table<double>(const DevPlan &P) { return P.w2_64; }
template <> __device__ __forceinline__ const float2 *w2_table<float>(const DevPlan &P) { return P.w2_32; }

// 8-byte asynchronous global -> shared copy (completes at cp_async_wait_all).
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst))),
                 "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst))),
                 "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// Factor N into radices: 8s first, then 4, 2, 3, 5, then remaining primes.
__device__ int factorize(int N, int *rad)
{
    int np = 0;
    while (N % 8 == 0) { rad[np++] = 8; N /= 8; }
    while (N % 4 == 0) { rad[np++] = 4; N /= 4; }
    while (N % 2 == 0) { rad[np++] = 2; N /= 2; }
    while (N % 3 == 0) { rad[np++] = 3; N /= 3; }
    while (N % 5 == 0) { rad[np++] = 5; N /= 5; }
    for (int p = 7; N > 1; p += 2) {
        while (N % p == 0) { rad[np++] = p; N /= p; }
        if (p * p > N && N > 1) { rad[np++] = N; N = 1; }
    }
    return np;
}

// Self-sorting (Stockham) mixed-radix complex DFT of length N in shared
// memory, ping-ponging between src and dst; returns the buffer holding the
// result.  INV: sign + (inverse, unnormalised) or - (forward).  W is the
// shared-memory table w_N^q = e^{2 pi i q / N}, q < N (conjugated for the
// forward sign).  Pass with radix R and sub-transform size Ns:
//   Y[(j/Ns) Ns R + j%Ns + q Ns] = sum_r X[j + r N/R] w_{Ns R}^{r (j%Ns)} w_R^{r q}.
// WG: W is a global table read through the read-only cache with element
// stride wst (w_N^q = W[q wst]) instead of a shared-memory table.
// PAD: the buffers hold element i at i + i / 16 (one unused slot per 16
// elements), which makes the strided stores of the first passes free of
// shared-memory bank conflicts.
template <bool INV, typename R, typename C, int G = 1, bool WG = false, int NT = kThreads, bool PAD = false>
__device__ C *stockham(C *src, C *dst, const int N, const C *W, const int *rad, const int npass, const int gs = 0,
                      const int wst = 1)
{
    auto PI = [](int i) { return PAD ? i + (i >> 4) : i; };
    const int tid = threadIdx.x;
    const R sg = INV ? (R)1 : (R)-1;
    auto tw = [&](int q) {
        C w = WG ? __ldg(W + q * wst) : W[q];
        if (!INV) w.y = -w.y;
        return w;
    };
    // multiply by sg * i
    auto muli = [&](C a) {
        C c;
        c.x = -sg * a.y;
        c.y = sg * a.x;
        return c;
    };
    int Ns = 1;
    for (int pi = 0; pi < npass; ++pi) {
        const int Rr = rad[pi];
        const int NR = N / Rr;
        const int tscale = N / (Ns * Rr);  // w_{Ns R}^e = w_N^{e tscale}
        // j / Ns: a shift while Ns is a power of two (all earlier radices 8, 4, 2)
        const bool ns_pow2 = (Ns & (Ns - 1)) == 0;
        const int ns_sh = __ffs(Ns) - 1;
        // (g, kk) = (j / Ns, j % Ns) for j = tid, advanced by (dq, dr) per NT
        const int g0 = ns_pow2 ? (tid >> ns_sh) : tid / Ns;
        const int kk0 = tid - g0 * Ns;
        const int dq = ns_pow2 ? (NT >> ns_sh) : NT / Ns;
        const int dr = NT - dq * Ns;
        // Each butterfly loads the inputs of all G maps first and loads its
        // twiddles once for all of them; r kk tscale < R Ns N / (Ns R) = N,
        // so twiddle indices need no reduction.
        if (Rr == 8) {
            const R c8 = (R)0.70710678118654752440084436210485;  // 1/sqrt(2)
            int g = g0, kk = kk0;
            for (int j = tid; j < NR; j += NT, kk += dr, g += dq) {
                if (kk >= Ns) {
                    kk -= Ns;
                    ++g;
                }
                C v[G][8], w[8];
#pragma unroll
                for (int gm = 0; gm < G; ++gm)
#pragma unroll
                    for (int r = 0; r < 8; ++r) v[gm][r] = src[gm * gs + PI(j + r * NR)];
                if (kk) {
                    const int e = kk * tscale;
#pragma unroll
                    for (int r = 1; r < 8; ++r) w[r] = tw(r * e);
                }
                const int o = g * Ns * 8 + kk;
#pragma unroll
                for (int gm = 0; gm < G; ++gm) {
                    if (kk) {
#pragma unroll
                        for (int r = 1; r < 8; ++r) v[gm][r] = cmul(v[gm][r], w[r]);
                    }
                    // X_{2q} = DFT4(v_r + v_{r+4}), X_{2q+1} = DFT4((v_r - v_{r+4}) w8^r), w8 = e^{sg 2 pi i / 8}
                    C a[4], b[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        a[r] = cadd(v[gm][r], v[gm][r + 4]);
                        b[r] = csub(v[gm][r], v[gm][r + 4]);
                    }
                    b[1] = mk<R>(rmul(c8, b[1].x - sg * b[1].y), rmul(c8, b[1].y + sg * b[1].x));
                    b[2] = muli(b[2]);
                    b[3] = mk<R>(rmul(c8, -b[3].x - sg * b[3].y), rmul(c8, sg * b[3].x - b[3].y));
                    C *d = dst + gm * gs;
                    {
                        const C s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
                        const C s13 = cadd(a[1], a[3]), d13 = muli(csub(a[1], a[3]));
                        d[PI(o)] = cadd(s02, s13);
                        d[PI(o + 2 * Ns)] = cadd(d02, d13);
                        d[PI(o + 4 * Ns)] = csub(s02, s13);
                        d[PI(o + 6 * Ns)] = csub(d02, d13);
                    }
                    {
                        const C s02 = cadd(b[0], b[2]), d02 = csub(b[0], b[2]);
                        const C s13 = cadd(b[1], b[3]), d13 = muli(csub(b[1], b[3]));
                        d[PI(o + Ns)] = cadd(s02, s13);
                        d[PI(o + 3 * Ns)] = cadd(d02, d13);
                        d[PI(o + 5 * Ns)] = csub(s02, s13);
                        d[PI(o + 7 * Ns)] = csub(d02, d13);
                    }
                }
            }
        } else if (Rr == 2) {
            int g = g0, kk = kk0;
            for (int j = tid; j < NR; j += NT, kk += dr, g += dq) {
                if (kk >= Ns) {
                    kk -= Ns;
                    ++g;
                }
                C v[G][2];
#pragma unroll
                for (int gm = 0; gm < G; ++gm) {
                    v[gm][0] = src[gm * gs + PI(j)];
                    v[gm][1] = src[gm * gs + PI(j + NR)];
                }
                const C w1 = kk ? tw(kk * tscale) : mk<R>(1, 0);
                const int o = g * Ns * 2 + kk;
#pragma unroll
                for (int gm = 0; gm < G; ++gm) {
                    const C v1 = kk ? cmul(v[gm][1], w1) : v[gm][1];
                    C *d = dst + gm * gs;
                    d[PI(o)] = cadd(v[gm][0], v1);
                    d[PI(o + Ns)] = csub(v[gm][0], v1);
                }
            }
        } else if (Rr == 4) {
            int g = g0, kk = kk0;
            for (int j = tid; j < NR; j += NT, kk += dr, g += dq) {
                if (kk >= Ns) {
                    kk -= Ns;
                    ++g;
                }
                C v[G][4], w[4];
#pragma unroll
                for (int gm = 0; gm < G; ++gm)
#pragma unroll
                    for (int r = 0; r < 4; ++r) v[gm][r] = src[gm * gs + PI(j + r * NR)];
                if (kk) {
                    const int e = kk * tscale;
#pragma unroll
                    for (int r = 1; r < 4; ++r) w[r] = tw(r * e);
                }
                const int o = g * Ns * 4 + kk;
#pragma unroll
                for (int gm = 0; gm < G; ++gm) {
                    if (kk) {
#pragma unroll
                        for (int r = 1; r < 4; ++r) v[gm][r] = cmul(v[gm][r], w[r]);
                    }
                    // radix 4 with w_4 = sg * i
                    const C a0 = cadd(v[gm][0], v[gm][2]), a1 = csub(v[gm][0], v[gm][2]);
                    const C a2 = cadd(v[gm][1], v[gm][3]), a3 = muli(csub(v[gm][1], v[gm][3]));
                    C *d = dst + gm * gs;
                    d[PI(o)] = cadd(a0, a2);
                    d[PI(o + Ns)] = cadd(a1, a3);
                    d[PI(o + 2 * Ns)] = csub(a0, a2);
                    d[PI(o + 3 * Ns)] = csub(a1, a3);
                }
            }
        } else if (Rr == 3) {
            const R c3 = (R)-0.5;
            const R s3 = sg * (R)0.86602540378443864676372317075294;  // sg sin(2 pi / 3)
            int g = g0, kk = kk0;
            for (int j = tid; j < NR; j += NT, kk += dr, g += dq) {
                if (kk >= Ns) {
                    kk -= Ns;
                    ++g;
                }
                C v[G][3], w[3];
#pragma unroll
                for (int gm = 0; gm < G; ++gm)
#pragma unroll
                    for (int r = 0; r < 3; ++r) v[gm][r] = src[gm * gs + PI(j + r * NR)];
                if (kk) {
                    const int e = kk * tscale;
                    w[1] = tw(e);
                    w[2] = tw(2 * e);
                }
                const int o = g * Ns * 3 + kk;
#pragma unroll
                for (int gm = 0; gm < G; ++gm) {
                    if (kk) {
                        v[gm][1] = cmul(v[gm][1], w[1]);
                        v[gm][2] = cmul(v[gm][2], w[2]);
                    }
                    const C t1 = cadd(v[gm][1], v[gm][2]);
                    const C t2 = csub(v[gm][1], v[gm][2]);
                    const C m1 = mk<R>(rfma(c3, t1.x, v[gm][0].x), rfma(c3, t1.y, v[gm][0].y));
                    const C m2 = mk<R>(-rmul(s3, t2.y), rmul(s3, t2.x));  // i s3 (v1 - v2)
                    C *d = dst + gm * gs;
                    d[PI(o)] = cadd(v[gm][0], t1);
                    d[PI(o + Ns)] = cadd(m1, m2);
                    d[PI(o + 2 * Ns)] = csub(m1, m2);
                }
            }
        } else if (Rr == 5) {
            const R c1 = (R)0.30901699437494742410229341718282;        // cos(2 pi / 5)
            const R c2 = (R)-0.80901699437494742410229341718282;       // cos(4 pi / 5)
            const R s1 = sg * (R)0.95105651629515357211643933337938;   // sg sin(2 pi / 5)
            const R s2 = sg * (R)0.58778525229247312916870595463907;   // sg sin(4 pi / 5)
            int g = g0, kk = kk0;
            for (int j = tid; j < NR; j += NT, kk += dr, g += dq) {
                if (kk >= Ns) {
                    kk -= Ns;
                    ++g;
                }
                C v[G][5], w[5];
#pragma unroll
                for (int gm = 0; gm < G; ++gm)
#pragma unroll
                    for (int r = 0; r < 5; ++r) v[gm][r] = src[gm * gs + PI(j + r * NR)];
                if (kk) {
                    const int e = kk * tscale;
#pragma unroll
                    for (int r = 1; r < 5; ++r) w[r] = tw(r * e);
                }
                const int o = g * Ns * 5 + kk;
#pragma unroll
                for (int gm = 0; gm < G; ++gm) {
                    if (kk) {
#pragma unroll
                        for (int r = 1; r < 5; ++r) v[gm][r] = cmul(v[gm][r], w[r]);
                    }
                    const C a1 = cadd(v[gm][1], v[gm][4]), b1 = csub(v[gm][1], v[gm][4]);
                    const C a2 = cadd(v[gm][2], v[gm][3]), b2 = csub(v[gm][2], v[gm][3]);
                    const C v0 = v[gm][0];
                    const C m1 = mk<R>(rfma(c2, a2.x, rfma(c1, a1.x, v0.x)), rfma(c2, a2.y, rfma(c1, a1.y, v0.y)));
                    const C m2 = mk<R>(rfma(c1, a2.x, rfma(c2, a1.x, v0.x)), rfma(c1, a2.y, rfma(c2, a1.y, v0.y)));
                    // i (s1 b1 + s2 b2) and i (s2 b1 - s1 b2)
                    const C n1 = mk<R>(-rfma(s1, b1.y, rmul(s2, b2.y)), rfma(s1, b1.x, rmul(s2, b2.x)));
                    const C n2 = mk<R>(-rfma(s2, b1.y, -rmul(s1, b2.y)), rfma(s2, b1.x, -rmul(s1, b2.x)));
                    C *d = dst + gm * gs;
                    d[PI(o)] = cadd(v0, cadd(a1, a2));
                    d[PI(o + Ns)] = cadd(m1, n1);
                    d[PI(o + 2 * Ns)] = cadd(m2, n2);
                    d[PI(o + 3 * Ns)] = csub(m2, n2);
                    d[PI(o + 4 * Ns)] = csub(m1, n1);
                }
            }
        } else {
            // direct pass for a general prime radix: one thread per output,
            // Y[o + q Ns] = sum_r X[j + r NR] w_N^{r (kk tscale + q NR)}
            for (int t = tid; t < N; t += NT) {
                const int q = t / NR;
                const int j = t - q * NR;
                const int g = ns_pow2 ? (j >> ns_sh) : j / Ns;
                const int kk = j - g * Ns;
                const int e = kk * tscale + q * NR;  // < N
#pragma unroll
                for (int gm = 0; gm < G; ++gm) {
                    const C *sx = src + gm * gs;
                    C acc = sx[PI(j)];
                    int idx = e;
                    for (int rr = 1; rr < Rr; ++rr) {
                        acc = cadd(acc, cmul(sx[PI(j + rr * NR)], tw(idx)));
                        idx += e;
                        if (idx >= N) idx -= N;
                    }
                    dst[gm * gs + PI(g * Ns * Rr + kk + q * Ns)] = acc;
                }
            }
        }
        __syncthreads();
        C *tmp = src;
        src = dst;
        dst = tmp;
        Ns *= Rr;
    }
    return src;
}

// Bluestein's DFT of length N (sign + if INV) of x in a[0..N): with the
// chirp c_j = e^{sg i pi j^2 / N} (j^2 reduced mod 2N, read from the ring's
// table T[q] = e^{i pi q / n}, n = 2N or N), X_k = c_k sum_j (x_j c_j) conj(c_{k-j}),
// a circular convolution of length Mb >= 2N - 1 done as
// IFFT_Mb(FFT_Mb(x c) * Bh) with Bh = FFT_Mb(e^{-i pi t^2 / N}, wrapped) / Mb
// from the plan (the forward sign uses conj(Bh[-k])).  a and b hold Mb
// elements; W2 is w_Mb^q, q < Mb.  Returns the buffer holding X[0..N).
// The chirp c_j = e^{sg i pi j^2 / N} (sg = + for INV) from the ring's table
// T[q] = e^{i pi q / n}: c_j = T[(j^2 mod 2N) n / N]; j < Mb <= 4096, so j^2
// does not overflow.
template <bool INV, typename C>
__device__ __forceinline__ C blue_chirp(const C *__restrict__ T, int n, int N, int j)
{
    C c = T[((j * j) % (2 * N)) * (n / N)];
    if (!INV) c.y = -c.y;
    return c;
}

// PRE_POST = false: the caller has already multiplied x by the chirp (and
// zero-filled a[N..Mb)), and multiplies the result by the chirp itself.
template <bool INV, typename R, typename C, int G = 1, bool WG = false, int NT = kThreads, bool PRE_POST = true,
          bool PAD = false>
__device__ C *bluestein(C *a, C *b, const C *W2, const C *__restrict__ Bh, const C *__restrict__ T, int n, int N,
                        int Mb, const int *rad2, int np2, const int gs = 0, const int wst = 1)
{
    const int tid = threadIdx.x;
    auto chirp = [&](int j) { return blue_chirp<INV>(T, n, N, j); };
    auto PI = [](int i) { return PAD ? i + (i >> 4) : i; };
    if (PRE_POST) {
        for (int j = tid; j < Mb; j += NT) {
            const C c = (j < N) ? chirp(j) : mk<R>(0, 0);
#pragma unroll
            for (int gm = 0; gm < G; ++gm) {
                C *ax = a + (size_t)gm * gs;
                ax[PI(j)] = (j < N) ? cmul(ax[PI(j)], c) : c;
            }
        }
        __syncthreads();
    }
    C *f = stockham<false, R, C, G, WG, NT, PAD>(a, b, Mb, W2, rad2, np2, gs, wst);
    for (int k = tid; k < Mb; k += NT) {
        const C h = INV ? Bh[k] : cconj(Bh[k == 0 ? 0 : Mb - k]);
#pragma unroll
        for (int gm = 0; gm < G; ++gm) {
            C *fx = f + (size_t)gm * gs;
            fx[PI(k)] = cmul(fx[PI(k)], h);
        }
    }
    __syncthreads();
    C *y = stockham<true, R, C, G, WG, NT, PAD>(f, (f == a) ? b : a, Mb, W2, rad2, np2, gs, wst);
    if (PRE_POST) {
        for (int k = tid; k < N; k += NT) {
            const C c = chirp(k);
#pragma unroll
            for (int gm = 0; gm < G; ++gm) {
                C *yx = y + (size_t)gm * gs;
                yx[PI(k)] = cmul(yx[PI(k)], c);
            }
        }
        __syncthreads();
    }
    return y;
}

// Synthesis of ring r of plan P for maps [b_begin, b_end): delta is the
// plan's Delta array [map][ring][m], map the first pixel of map 0.  smem
// holds three buffers of cap complex elements.  All threads of the CTA call it.
template <typename R, bool BLUE>
__device__ __forceinline__ void ring_synth_body(const DevPlan &P, int r, const typename C2T<R>::type *__restrict__ delta,
                                                R *__restrict__ map, int b_begin, int b_end, int cap,
                                                unsigned char *smem_raw, int *s_rad, int *s_np_ptr)
{
    using C = typename C2T<R>::type;
    C *buf0 = reinterpret_cast<C *>(smem_raw);
    C *buf1 = buf0 + cap;
    C *W = buf1 + cap;  // w_N^q, q < N (direct) or w_Mb^q, q < Mb (Bluestein)
    int &s_np = *s_np_ptr;
    const int tid = threadIdx.x;
    const int n = P.nphi[r];
    const int M = P.mmax;
    const C *T = tw_table<R>(P) + P.twofs[r];  // T[q] = e^{i pi q / n}, q < 2n
    const int ps = P.ps[r];
    const double phi0 = P.phi0[r];
    const bool even = (n % 2) == 0;
    const int N = even ? n / 2 : n;                     // complex DFT length
    const int nb = even ? n / 2 + 1 : (n - 1) / 2 + 1;  // half-spectrum bins
    const int tstep = even ? 4 : 2;                     // T index of w_N^1
    const int Mb = BLUE ? P.blue_mb[r] : 0;
    const C *Bh = BLUE ? bhat_table<R>(P) + P.blue_ofs[r] : nullptr;

    if (BLUE) {
        if (tid == 0) s_np = factorize(Mb, s_rad);
        const C *w2 = w2_table<R>(P);
        const int wstep = kBlueMaxMb / Mb;
        for (int q = tid; q < Mb; q += kThreads) W[q] = w2[q * wstep];
    } else {
        if (tid == 0) s_np = factorize(N, s_rad);
        for (int q = tid; q < N; q += kThreads) W[q] = T[q * tstep];
    }

    for (int b = b_begin; b < b_end; ++b) {
        const size_t row = P.ring_row ? (size_t)b * P.delta_rows + SHT_IDX(P.dbg, P.ring_row[r], P.delta_rows, 201)
                                      : (size_t)b * P.nrings + r;
        const C *D = delta + row * (size_t)(M + 1);
        // 1. phase shift + fold onto the half spectrum, into buf1[0..nb);
        //    the phase index (m ps) mod 2n advances by (n ps) mod 2n along m = k, k + n, ...
        const int pstep = (ps >= 0) ? (int)(((long long)n * ps) % (2 * n)) : 0;
        for (int k = tid; k < nb; k += kThreads) {
            C acc = mk<R>(0, 0);
            int pi = (ps >= 0) ? (int)(((long long)k * ps) % (2 * n)) : 0;
            for (int m = k; m <= M; m += n) {
                C ph;
                if (ps >= 0) {
                    ph = T[pi];
                    pi += pstep;
                    if (pi >= 2 * n) pi -= 2 * n;
                } else {
                    double sn, cs;
                    sincos((double)m * phi0, &sn, &cs);
                    ph = mk<R>((R)cs, (R)sn);
                }
                acc = cadd(acc, cmul(D[m], ph));
            }
            pi = (ps >= 0) ? (int)(((long long)(n - k) * ps) % (2 * n)) : 0;
            for (int m = n - k; m <= M; m += n) {
                C ph;
                if (ps >= 0) {
                    ph = T[pi];
                    pi += pstep;
                    if (pi >= 2 * n) pi -= 2 * n;
                } else {
                    double sn, cs;
                    sincos((double)m * phi0, &sn, &cs);
                    ph = mk<R>((R)cs, (R)sn);
                }
                if (m >= 1) acc = cadd(acc, cconj(cmul(D[m], ph)));
            }
            buf1[k] = acc;
        }
        __syncthreads();

        // 2. spectrum of the complex DFT, into buf0[0..N)
        if (even) {
            for (int k = tid; k < N; k += kThreads) {
                const C f = buf1[k];
                const C g = cconj(buf1[N - k]);
                const C w = T[2 * k];  // e^{2 pi i k / n}
                buf0[k] = cadd(cadd(f, g), cmuli(cmul(w, csub(f, g))));
            }
        } else {
            for (int k = tid; k < N; k += kThreads) buf0[k] = (k < nb) ? buf1[k] : cconj(buf1[N - k]);
        }
        __syncthreads();

        // 3. inverse complex DFT of length N
        C *src = BLUE ? bluestein<true, R>(buf0, buf1, W, Bh, T, n, N, Mb, s_rad, s_np)
                      : stockham<true, R>(buf0, buf1, N, W, s_rad, s_np);

        // 4. store the ring
        SHT_CHECK(P.dbg, P.ofs[r] + n <= P.npix, 202);
        R *out = map + (size_t)b * P.npix + P.ofs[r];
        if (even) {
            for (int j = tid; j < N; j += kThreads) {
                const C z = src[j];
                out[2 * j] = z.x;
                out[2 * j + 1] = z.y;
            }
        } else {
            for (int j = tid; j < N; j += kThreads) out[j] = src[j].x;
        }
        __syncthreads();
    }
}

template <typename R, bool BLUE>
__global__ void __launch_bounds__(kThreads)
ring_synth_kernel(const __grid_constant__ DevPlan P, const typename C2T<R>::type *__restrict__ delta,
                  R *__restrict__ map, int nmaps, int gmaps)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_rad[32];
    __shared__ int s_np;
    const int r = BLUE ? P.rings_blue[blockIdx.x] : P.rings_smooth[blockIdx.x];
    ring_synth_body<R, BLUE>(P, r, delta, map, blockIdx.y * gmaps, min(nmaps, (int)(blockIdx.y + 1) * gmaps),
                             BLUE ? P.blue_cap : P.fft_cap, smem_raw, s_rad, &s_np);
}

// FP32 ring step of the tensor-core forms, reading Delta in the layout the
// tensor-core Legendre kernels write, [ring][m][map] for nmaps maps.  CTA
// (ring, map group) synthesises G consecutive maps of one ring together: the
// fold reads the G maps' Delta_m side by side (one sector per m for G = 4)
// and shares the phase factors, and every FFT pass handles all G maps between
// two barriers.  Shared memory: two regions of G buffers of cap complex
// elements (A: folded spectra, B: DFT inputs; the DFT ping-pongs between
// them).  The ring's Delta block (M + 1 orders x G maps) is first copied into
// region B by asynchronous copies, all in flight at once, so that the fold
// reads shared memory instead of paying a global-memory latency per bin (when
// M + 1 > cap the fold reads global memory directly).  CTAs of one ring are adjacent in the grid
// (block = ring index x groups + group), so the maps of a sector are read at
// about the same time.  The twiddles come from the plan's global tables
// through the read-only cache, which leaves shared memory to the buffers.
// MULTI: block i synthesises ring mitems[i].y of request mitems[i].x (one map,
// G = 1) with that request's plan, Delta and map; capm is the buffer size the
// launch's shared memory was sized for.
template <bool BLUE, int G, int NT, bool MULTI = false>
__global__ void __launch_bounds__(NT, (NT == 256 && G <= 2) ? 3 : 1)
ring_synth_mf_kernel(const __grid_constant__ DevPlan P0, const float2 *__restrict__ delta0, float *__restrict__ map0,
                     int nmaps0, const DevPlan *__restrict__ plans, const int2 *__restrict__ mitems,
                     const __grid_constant__ MultiTcPtrs mp, int capm)
{
    using R = float;
    using C = float2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_rad[32];
    __shared__ int s_np;
    int li, b0, req = 0;
    if constexpr (MULTI) {
        const int2 w = mitems[blockIdx.x];
        req = w.x;
        li = w.y;
        b0 = 0;
    } else {
        const int ngroups = (nmaps0 + G - 1) / G;
        li = blockIdx.x / ngroups;
        b0 = (blockIdx.x - li * ngroups) * G;
    }
    const DevPlan &P = MULTI ? plans[req] : P0;
    const float2 *__restrict__ delta = MULTI ? static_cast<const float2 *>(mp.delta[req]) : delta0;
    float *__restrict__ map = MULTI ? static_cast<float *>(mp.map[req]) : map0;
    const int nmaps = MULTI ? 1 : nmaps0;
    const int gn = min(G, nmaps - b0);  // maps in this CTA
    const int r = MULTI ? li : (BLUE ? P.rings_blue[li] : P.rings_smooth[li]);
    const int cap = MULTI ? capm : (BLUE ? P.blue_cap : P.fft_cap);
    const int capP = cap + (cap >> 4) + 1;      // padded buffer (element i at i + i / 16)
    auto PI = [](int i) { return i + (i >> 4); };
    C *A0 = reinterpret_cast<C *>(smem_raw);  // map g: A at A0 + g capP, B at A0 + (G + g) capP
    C *B0 = A0 + G * capP;
    const int gs = capP;
    const int tid = threadIdx.x;
    const int n = P.nphi[r];
    const int M = ring_mtop(P, r);  // Delta_m is zero past it (never read)
    const C *T = tw_table<R>(P) + P.twofs[r];  // T[q] = e^{i pi q / n}, q < 2n
    const int ps = P.ps[r];
    const double phi0 = P.phi0[r];
    const bool even = (n % 2) == 0;
    const int N = even ? n / 2 : n;
    const int nb = even ? n / 2 + 1 : (n - 1) / 2 + 1;
    const int tstep = even ? 4 : 2;
    const int Mb = BLUE ? P.blue_mb[r] : 0;
    const C *Cp = BLUE ? P.chirp32 + P.chirp_ofs[r] : nullptr;  // e^{i pi t^2 / N}, t < N

    if (tid == 0) s_np = factorize(BLUE ? Mb : N, s_rad);

    // 1. phase shift + fold of the gn maps onto the half spectrum, into A_g[0..nb):
    //    F_k = sum_{m = k mod n} Delta_m e^{i m phi0} + sum_{m >= 1, -m = k mod n} conj(...)
    SHT_CHECK(P.dbg, r >= 0 && r < P.nrings && b0 + gn <= nmaps, 203);
    SHT_CHECK(P.dbg, !(M + 1 <= cap) || (size_t)G * (M + 1) <= (size_t)G * capP, 204);
    const C *D = delta + (size_t)r * (P.mmax + 1) * nmaps + b0;  // D[m nmaps + g]
    const bool staged = M + 1 <= cap;
    const int n2 = 2 * n;
    // Phase indices (m ps) mod 2n advance incrementally: bin k starts at k ps, the
    // next bin of the thread at (k + NT) ps, the next alias m + n at m ps + n ps.
    const int pstep = (ps >= 0) ? (n * ps) % n2 : 0;
    const int dpk = (ps >= 0) ? (NT * ps) % n2 : 0;
    if (staged) {
        // Delta_m of map g -> B0[m G + g] by asynchronous copies, all in flight at
        // once (16 bytes = two maps per copy when aligned)
        const bool v16 = G >= 2 && gn == G && (nmaps & 1) == 0 && (b0 & 1) == 0;
        const C *src = D + (size_t)tid * nmaps;
        for (int m = tid; m <= M; m += NT, src += (size_t)NT * nmaps) {
            if (v16) {
#pragma unroll
                for (int h = 0; h < G; h += 2) cp_async16(&B0[m * G + h], src + h);
            } else {
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    if (g < gn)
                        cp_async8(&B0[m * G + g], src + g);
                    else
                        B0[m * G + g] = mk<R>(0, 0);
                }
            }
        }
        // the phase of each of the thread's bins' first alias (m = k), loaded
        // while the copies are in flight; bins k = tid + j NT, j < JB, cover
        // nb <= cap <= 4097
        constexpr int JB = 4352 / NT + 1;
        C ph0[JB];
        int pk0[JB];
        {
            int pk = (ps >= 0) ? (tid * ps) % n2 : 0;
#pragma unroll
            for (int j = 0; j < JB; ++j) {
                const int k = tid + j * NT;
                pk0[j] = pk;
                if (k < nb && k <= M) {
                    if (ps >= 0) {
                        ph0[j] = T[pk];
                    } else {
                        double sn, cs;
                        sincos((double)k * phi0, &sn, &cs);
                        ph0[j] = mk<R>((R)cs, (R)sn);
                    }
                }
                pk += dpk;
                if (pk >= n2) pk -= n2;
            }
        }
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int j = 0; j < JB; ++j) {
            const int k = tid + j * NT;
            if (k >= nb) break;
            C acc[G];
#pragma unroll
            for (int g = 0; g < G; ++g) acc[g] = mk<R>(0, 0);
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
                // pass 0: m = k + j n; pass 1: m = n - k + j n (>= 1), conjugated
                const int pk = pk0[j];
                const int m0 = pass == 0 ? k : n - k;
                int pi = pass == 0 ? pk : pstep - pk + (pstep < pk ? n2 : 0);
                for (int m = m0; m <= M; m += n) {
                    C ph;
                    if (pass == 0 && m == k) {
                        ph = ph0[j];
                    } else if (ps >= 0) {
                        ph = T[pi];
                    } else {
                        double sn, cs;
                        sincos((double)m * phi0, &sn, &cs);
                        ph = mk<R>((R)cs, (R)sn);
                    }
                    pi += pstep;
                    if (pi >= n2) pi -= n2;
                    if (pass == 1 && m < 1) continue;
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const C v = cmul(B0[m * G + g], ph);
                        acc[g] = cadd(acc[g], pass == 0 ? v : cconj(v));
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g)
                if (g < gn) A0[g * capP + PI(k)] = acc[g];
        }
    } else {
        // Delta too long to stage: Delta from global memory
        int pk = (ps >= 0) ? (tid * ps) % n2 : 0;
        for (int k = tid; k < nb; k += NT) {
            C acc[G];
#pragma unroll
            for (int g = 0; g < G; ++g) acc[g] = mk<R>(0, 0);
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
                const int m0 = pass == 0 ? k : n - k;
                int pi = pass == 0 ? pk : pstep - pk + (pstep < pk ? n2 : 0);
                for (int m = m0; m <= M; m += n) {
                    C ph;
                    if (ps >= 0) {
                        ph = T[pi];
                        pi += pstep;
                        if (pi >= n2) pi -= n2;
                    } else {
                        double sn, cs;
                        sincos((double)m * phi0, &sn, &cs);
                        ph = mk<R>((R)cs, (R)sn);
                    }
                    if (pass == 1 && m < 1) continue;
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        if (g < gn) {
                            const C v = cmul(D[(size_t)m * nmaps + g], ph);
                            acc[g] = cadd(acc[g], pass == 0 ? v : cconj(v));
                        }
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g)
                if (g < gn) A0[g * capP + PI(k)] = acc[g];
            pk += dpk;
            if (pk >= n2) pk -= n2;
        }
    }
    __syncthreads();

    // 2. spectrum of the complex DFT, into B_g[0..N)
    //    (Bluestein rings: times the chirp, and zero up to the convolution length Mb)
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const C *F = A0 + g * capP;
        C *Bg = B0 + g * capP;
#pragma unroll 4
        for (int k = tid; k < N; k += NT) {
            C z;
            if (even) {
                const C f = F[PI(k)];
                const C h = cconj(F[PI(N - k)]);
                const C w = T[2 * k];  // e^{2 pi i k / n}
                z = cadd(cadd(f, h), cmuli(cmul(w, csub(f, h))));
            } else {
                z = (k < nb) ? F[PI(k)] : cconj(F[PI(N - k)]);
            }
            Bg[PI(k)] = BLUE ? cmul(z, Cp[k]) : z;
        }
        if (BLUE)
            for (int k = N + tid; k < Mb; k += NT) Bg[PI(k)] = mk<R>(0, 0);
    }
    __syncthreads();

    // 3. inverse complex DFT of length N of every map
    // (a CTA holding fewer than G maps transforms its spare buffers too,
    // harmlessly, and never stores them)
    C *src = BLUE ? bluestein<true, R, C, G, true, NT, false, true>(B0, A0, w2_table<R>(P), bhat_table<R>(P) + P.blue_ofs[r], T, n,
                                                       N, Mb, s_rad, s_np, gs, Mb > 0 ? kBlueMaxMb / Mb : 1)
                  : stockham<true, R, C, G, true, NT, true>(B0, A0, N, T, s_rad, s_np, gs, tstep);

    // 4. store the rings (Bluestein rings: times the chirp; even n: pixel pairs
    //    as one 8-byte store when aligned)
    SHT_CHECK(P.dbg, P.ofs[r] + n <= P.npix, 205);
    for (int g = 0; g < gn; ++g) {
        const C *z = src + g * gs;
        R *out = map + (size_t)(b0 + g) * P.npix + P.ofs[r];
        auto val = [&](int j) { return BLUE ? cmul(z[PI(j)], Cp[j]) : z[PI(j)]; };
        if (even && (reinterpret_cast<uintptr_t>(out) & 7) == 0) {
            float2 *o2 = reinterpret_cast<float2 *>(out);
#pragma unroll 4
            for (int j = tid; j < N; j += NT) o2[j] = val(j);
        } else if (even) {
            for (int j = tid; j < N; j += NT) {
                const C v = val(j);
                out[2 * j] = v.x;
                out[2 * j + 1] = v.y;
            }
        } else {
            for (int j = tid; j < N; j += NT) out[j] = val(j).x;
        }
    }
}

// Ring step of many one-map requests: CTA i synthesises ring items[i].y of
// request items[i].x; cap is the largest buffer over the requests.
template <typename R, bool BLUE>
__global__ void __launch_bounds__(kThreads)
ring_synth_multi_kernel(const DevPlan *__restrict__ plans, const int2 *__restrict__ items, const MultiPtrs ptrs,
                        int cap)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_rad[32];
    __shared__ int s_np;
    const int2 w = items[blockIdx.x];
    ring_synth_body<R, BLUE>(plans[w.x], w.y, static_cast<const typename C2T<R>::type *>(ptrs.delta[w.x]),
                             static_cast<R *>(ptrs.map[w.x]), 0, 1, cap, smem_raw, s_rad, &s_np);
}

// Ring step of the transpose (map2alm_adjoint): for every ring r and m <= M,
//   q_m(r) = sum_j y_rj e^{-i m (phi0_r + 2 pi j / n)} = e^{-i m phi0} Y_{m mod n},
// where Y is the forward real DFT of the ring (Y_{n-k} = conj Y_k).  For even
// n the real DFT runs as one complex DFT of z_j = y_{2j} + i y_{2j+1}, length
// h = n/2: Y_k = (Z_k + conj Z_{h-k})/2 - (i/2) w^{-k} (Z_k - conj Z_{h-k}).
// wring (optional): q_m(r) is multiplied by the ring's pixel quadrature weight.
template <typename R, bool BLUE>
__global__ void __launch_bounds__(kThreads)
ring_analysis_kernel(const DevPlan P, const R *__restrict__ map, typename C2T<R>::type *__restrict__ qout,
                     const double *__restrict__ wring, int nmaps, int gmaps)
{
    using C = typename C2T<R>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int cap = BLUE ? P.blue_cap : P.fft_cap;
    C *buf0 = reinterpret_cast<C *>(smem_raw);
    C *buf1 = buf0 + cap;
    C *W = buf1 + cap;
    __shared__ int s_rad[32];
    __shared__ int s_np;

    const int r = BLUE ? P.rings_blue[blockIdx.x] : P.rings_smooth[blockIdx.x];
    const int tid = threadIdx.x;
    const int n = P.nphi[r];
    const int M = P.mmax;
    const C *T = tw_table<R>(P) + P.twofs[r];
    const int ps = P.ps[r];
    const double phi0 = P.phi0[r];
    const bool even = (n % 2) == 0;
    const int N = even ? n / 2 : n;
    const int nb = even ? n / 2 + 1 : (n - 1) / 2 + 1;
    const int tstep = even ? 4 : 2;
    const int Mb = BLUE ? P.blue_mb[r] : 0;
    const C *Bh = BLUE ? bhat_table<R>(P) + P.blue_ofs[r] : nullptr;

    if (BLUE) {
        if (tid == 0) s_np = factorize(Mb, s_rad);
        const C *w2 = w2_table<R>(P);
        const int wstep = kBlueMaxMb / Mb;
        for (int q = tid; q < Mb; q += kThreads) W[q] = w2[q * wstep];
    } else {
        if (tid == 0) s_np = factorize(N, s_rad);
        for (int q = tid; q < N; q += kThreads) W[q] = T[q * tstep];
    }

    const int b_end = min(nmaps, (int)(blockIdx.y + 1) * gmaps);
    for (int b = blockIdx.y * gmaps; b < b_end; ++b) {
        const R *in = map + (size_t)b * P.npix + P.ofs[r];
        if (even) {
            for (int j = tid; j < N; j += kThreads) buf0[j] = mk<R>(in[2 * j], in[2 * j + 1]);
        } else {
            for (int j = tid; j < N; j += kThreads) buf0[j] = mk<R>(in[j], (R)0);
        }
        __syncthreads();

        C *res = BLUE ? bluestein<false, R>(buf0, buf1, W, Bh, T, n, N, Mb, s_rad, s_np)
                      : stockham<false, R>(buf0, buf1, N, W, s_rad, s_np);
        C *Y = (res == buf0) ? buf1 : buf0;
        if (even) {
            for (int k = tid; k < nb; k += kThreads) {
                const C z = res[k == N ? 0 : k];
                const C zc = cconj(res[k == 0 ? 0 : N - k]);
                C w = T[2 * k];  // e^{2 pi i k / n}; conjugated below
                w.y = -w.y;
                const C e = cadd(z, zc);
                const C o = cmul(w, csub(z, zc));
                // Y_k = e/2 - (i/2) o
                Y[k] = mk<R>((R)0.5 * (e.x + o.y), (R)0.5 * (e.y - o.x));
            }
        } else {
            for (int k = tid; k < nb; k += kThreads) Y[k] = res[k];
        }
        __syncthreads();

        C *q = qout + ((size_t)b * P.nrings + r) * (size_t)(M + 1);
        for (int m = tid; m <= M; m += kThreads) {
            const int k = m % n;
            const C yk = (k < nb) ? Y[k] : cconj(Y[n - k]);
            C ph;
            if (ps >= 0) {
                ph = T[(int)(((long long)m * ps) % (2 * n))];
            } else {
                double sn, cs;
                sincos((double)m * phi0, &sn, &cs);
                ph = mk<R>((R)cs, (R)sn);
            }
            const C v = cmul(yk, cconj(ph));
            q[m] = wring ? mk<R>(rmul(v.x, (R)wring[r]), rmul(v.y, (R)wring[r])) : v;
        }
        __syncthreads();
    }
}

// Launch one ring kernel over the smooth ring list and one over the
// Bluestein ring list (each with its own shared-memory size).
template <typename K, typename... Args>
cudaError_t launch_two(K smooth, K blue, const DevPlan &P, bool fp64, int nmaps, int group, cudaStream_t st,
                       Args... args)
{
    if (nmaps <= 0) return cudaSuccess;
    const int g = group > 0 ? std::min(group, nmaps) : ring_group(nmaps);
    const int gy = (nmaps + g - 1) / g;
    if (P.n_smooth > 0) {
        const size_t smem = ring_smem_bytes_for_cap(P.fft_cap, fp64);
        if (smem > 40 * 1024) {  // dynamic + static above the 48 KB default needs the opt-in
            cudaError_t e = cudaFuncSetAttribute(smooth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        smooth<<<dim3(P.n_smooth, gy), kThreads, smem, st>>>(P, args..., nmaps, g);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (P.n_blue > 0) {
        const size_t smem = ring_smem_bytes_for_cap(P.blue_cap, fp64);
        if (smem > 40 * 1024) {  // dynamic + static above the 48 KB default needs the opt-in
            cudaError_t e = cudaFuncSetAttribute(blue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        blue<<<dim3(P.n_blue, gy), kThreads, smem, st>>>(P, args..., nmaps, g);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace


cudaError_t launch_ring_synth_fp64(const DevPlan &P, const double2 *delta, double *map, int nmaps, int group,
                                   cudaStream_t st)
{
    return launch_two(ring_synth_kernel<double, false>, ring_synth_kernel<double, true>, P, true, nmaps, group, st,
                      delta, map);
}

cudaError_t launch_ring_synth_mf_multi(const DevPlan *plans_dev, const int2 *smooth_items, int n_smooth,
                                       int smooth_cap, const int2 *blue_items, int n_blue, int blue_cap,
                                       const MultiTcPtrs &mp, int nt, cudaStream_t st)
{
    const bool big = nt >= 512;
    for (int pass = 0; pass < 2; ++pass) {
        const bool blue = pass == 1;
        const int n = blue ? n_blue : n_smooth;
        if (n <= 0) continue;
        const int cap = blue ? blue_cap : smooth_cap;
        const size_t smem = ring_mf_smem_bytes(cap, 1);
        auto k = blue ? (big ? ring_synth_mf_kernel<true, 1, 512, true> : ring_synth_mf_kernel<true, 1, 256, true>)
                      : (big ? ring_synth_mf_kernel<false, 1, 512, true> : ring_synth_mf_kernel<false, 1, 256, true>);
        if (smem > 40 * 1024) {  // dynamic + static above the 48 KB default needs the opt-in
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k<<<n, big ? 512 : 256, smem, st>>>(DevPlan{}, nullptr, nullptr, 1, plans_dev, blue ? blue_items : smooth_items,
                                            mp, cap);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t ring_mf_smem_bytes(int cap, int G) { return (size_t)2 * G * (cap + (cap >> 4) + 1) * sizeof(float2); }

cudaError_t launch_ring_synth_mf(const DevPlan &P, const float2 *delta_rm, float *map, int nmaps, int g_smooth,
                                 int g_blue, int nt, cudaStream_t st)
{
    if (nmaps <= 0) return cudaSuccess;
    for (int pass = 0; pass < 2; ++pass) {
        const bool blue = pass == 1;
        const int nl = blue ? P.n_blue : P.n_smooth;
        if (nl <= 0) continue;
        const int cap = blue ? P.blue_cap : P.fft_cap;
        int G = std::max(1, std::min(blue ? g_blue : g_smooth, 4));
        if (G == 3) G = 2;
        while (G > 1 && ring_mf_smem_bytes(cap, G) > (size_t)227 * 1024) G /= 2;
        const size_t smem = ring_mf_smem_bytes(cap, G);
        using K = void (*)(const DevPlan, const float2 *, float *, int, const DevPlan *, const int2 *,
                           const MultiTcPtrs, int);
        const bool big = nt >= 512;
        K k = blue ? (G == 4   ? (big ? ring_synth_mf_kernel<true, 4, 512> : ring_synth_mf_kernel<true, 4, 256>)
                      : G == 2 ? (big ? ring_synth_mf_kernel<true, 2, 512> : ring_synth_mf_kernel<true, 2, 256>)
                               : (big ? ring_synth_mf_kernel<true, 1, 512> : ring_synth_mf_kernel<true, 1, 256>))
                   : (G == 4   ? (big ? ring_synth_mf_kernel<false, 4, 512> : ring_synth_mf_kernel<false, 4, 256>)
                      : G == 2 ? (big ? ring_synth_mf_kernel<false, 2, 512> : ring_synth_mf_kernel<false, 2, 256>)
                               : (big ? ring_synth_mf_kernel<false, 1, 512> : ring_synth_mf_kernel<false, 1, 256>));
        if (smem > 40 * 1024) {  // dynamic + static above the 48 KB default needs the opt-in
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        const long long nblk = (long long)nl * ((nmaps + G - 1) / G);
        static const MultiTcPtrs none{};
        k<<<(unsigned)nblk, big ? 512 : 256, smem, st>>>(P, delta_rm, map, nmaps, nullptr, nullptr, none, 0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_ring_synth_multi_fp64(const DevPlan *plans, const int2 *smooth_items, int n_smooth,
                                         int smooth_cap, const int2 *blue_items, int n_blue, int blue_cap,
                                         const MultiPtrs &ptrs, cudaStream_t st)
{
    if (n_smooth > 0) {
        auto k = ring_synth_multi_kernel<double, false>;
        const size_t smem = ring_smem_bytes_for_cap(smooth_cap, true);
        if (smem > 40 * 1024) {  // dynamic + static above the 48 KB default needs the opt-in
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k<<<n_smooth, kThreads, smem, st>>>(plans, smooth_items, ptrs, smooth_cap);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_blue > 0) {
        auto k = ring_synth_multi_kernel<double, true>;
        const size_t smem = ring_smem_bytes_for_cap(blue_cap, true);
        if (smem > 40 * 1024) {  // dynamic + static above the 48 KB default needs the opt-in
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k<<<n_blue, kThreads, smem, st>>>(plans, blue_items, ptrs, blue_cap);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_ring_analysis_fp64(const DevPlan &P, const double *map, double2 *q, int nmaps,
                                      const double *wring, cudaStream_t st)
{
    return launch_two(ring_analysis_kernel<double, false>, ring_analysis_kernel<double, true>, P, true, nmaps, 0, st,
                      map, q, wring);
}

cudaError_t launch_ring_analysis_fp32(const DevPlan &P, const float *map, float2 *q, int nmaps,
                                      const double *wring, int group, cudaStream_t st)
{
    return launch_two(ring_analysis_kernel<float, false>, ring_analysis_kernel<float, true>, P, false, nmaps, group,
                      st, map, q, wring);
}


}  // namespace sht
