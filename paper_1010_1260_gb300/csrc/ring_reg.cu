// FP32 ring step of the tensor-core forms (Eq. Delta2map, sec. 2.2.2), for
// even ring lengths n whose half-length N = n / 2 either is a power of two in
// [256, 4096] (direct transform of length L = N) or has N <= 2048 (Bluestein's
// algorithm with a power-of-two convolution length L = max(256, 2^ceil(log2(2N - 1)))).
// Per ring r and map:
//   1. phase shift and fold (the FFT "wrapping" of sec. 2.2.2):
//      F_k = sum_{m = k mod n} Delta_m e^{i m phi0} + sum_{m >= 1, m = -k mod n} conj(Delta_m e^{i m phi0});
//   2. the real inverse DFT of length n as one complex DFT of length N:
//      Z_k = (F_k + conj F_{N-k}) + i w^k (F_k - conj F_{N-k}), w = e^{2 pi i / n},
//      z = IDFT_N(Z), pixel 2j = Re z_j, pixel 2j + 1 = Im z_j;
//      Bluestein: IDFT_N(Z)_k = c_k IFFT_L(FFT_L(Z c) * Bh)_k with the chirp
//      c_t = e^{i pi t^2 / N} and Bh = FFT_L(conj chirp, wrapped) / L (plan tables).
//
// Design (one persistent launch over (ring, pair of maps) units, units listed
// by decreasing cost, unit u run by CTA u mod grid):
//   * the Delta block of a unit (M + 1 orders x 2 maps, 16 bytes per order) is
//     brought into one of two shared-memory slots two units ahead of its use,
//     by tensor-map bulk copies (cp.async.bulk.tensor, boxes of 256 orders)
//     completing on an mbarrier, or by 16/8-byte asynchronous copies where a
//     tensor map cannot describe the layout (odd map counts, the many-request
//     form); the slot is released as soon as the fold has read it, so every
//     copy overlaps the FFTs of the two units before it;
//   * the FFT runs in registers: L / 16 threads per map, 16 elements each, two
//     radix-16 passes and one radix-(L / 256) pass in Stockham order, with the
//     data exchanged through one padded shared-memory buffer between passes;
//     a CTA of 256 threads runs 4096 / L maps of the unit at once (both maps
//     one after the other when L = 4096);
//   * every product is an explicitly rounded multiply or fused multiply-add, so
//     the per-plan and many-request instantiations give identical bits.
#include "sht.h"
#include "sht_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

namespace sht {
namespace {

constexpr int kRT = 256;                 // threads per CTA
constexpr int kBoxRows = 256;            // orders per tensor-map box
constexpr int kXElems = 4096 + 4096 / 16;  // exchange buffer, padded (one slot per 16 elements)
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ int PX(int i) { return i + (i >> 4); }

__device__ __forceinline__ float2 c2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return c2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return c2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return c2(a.x, -a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return c2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
// times i, exact
__device__ __forceinline__ float2 cmuli(float2 a) { return c2(-a.y, a.x); }
// 4-point inverse DFT (sign +) in place.
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = cmuli(csub(a1, a3));
    a0 = cadd(t0, t2);
    a1 = cadd(t1, t3);
    a2 = csub(t0, t2);
    a3 = csub(t1, t3);
}

// 16-point inverse DFT, y[q] = sum_r x[r] e^{2 pi i r q / 16}: r = r1 + 4 r2,
// q = q1 + 4 q2; DFT4 over r2, twiddle w16^{r1 q1}, DFT4 over r1.
__device__ __forceinline__ void dft16(const float2 (&x)[16], float2 (&y)[16])
{
    constexpr float C1 = 0.92387953251128675613f;  // cos(pi/8)
    constexpr float S1 = 0.38268343236508977173f;  // sin(pi/8)
    constexpr float RH = 0.70710678118654752440f;  // cos(pi/4)
    float2 a[4][4];
#pragma unroll
    for (int r1 = 0; r1 < 4; ++r1) {
        a[r1][0] = x[r1];
        a[r1][1] = x[r1 + 4];
        a[r1][2] = x[r1 + 8];
        a[r1][3] = x[r1 + 12];
        dft4(a[r1][0], a[r1][1], a[r1][2], a[r1][3]);
    }
    // w16^e for e = r1 q1 in {1, 2, 3, 4, 6, 9}
    const float2 w1 = c2(C1, S1), w2 = c2(RH, RH), w3 = c2(S1, C1);
    const float2 w6 = c2(-RH, RH), w9 = c2(-C1, -S1);
    a[1][1] = cmul(a[1][1], w1);
    a[1][2] = cmul(a[1][2], w2);
    a[1][3] = cmul(a[1][3], w3);
    a[2][1] = cmul(a[2][1], w2);
    a[2][2] = cmuli(a[2][2]);
    a[2][3] = cmul(a[2][3], w6);
    a[3][1] = cmul(a[3][1], w3);
    a[3][2] = cmul(a[3][2], w6);
    a[3][3] = cmul(a[3][3], w9);
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1) {
        float2 b0 = a[0][q1], b1 = a[1][q1], b2 = a[2][q1], b3 = a[3][q1];
        dft4(b0, b1, b2, b3);
        y[q1] = b0;
        y[q1 + 4] = b1;
        y[q1 + 8] = b2;
        y[q1 + 12] = b3;
    }
}

// R-point inverse DFT (R = 2, 4, 8, 16) of v[0..R) in place, natural order out.
template <int R> __device__ __forceinline__ void dft_r(float2 (&v)[R]);
template <> __device__ __forceinline__ void dft_r<2>(float2 (&v)[2])
{
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
template <> __device__ __forceinline__ void dft_r<4>(float2 (&v)[4]) { dft4(v[0], v[1], v[2], v[3]); }
template <> __device__ __forceinline__ void dft_r<8>(float2 (&v)[8])
{
    // r = r1 + 2 r2: DFT4 over r2, twiddle w8^{r1 q1}, DFT2 over r1
    constexpr float RH = 0.70710678118654752440f;
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4(e0, e1, e2, e3);
    dft4(o0, o1, o2, o3);
    o1 = cmul(o1, c2(RH, RH));
    o2 = cmuli(o2);
    o3 = cmul(o3, c2(-RH, RH));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}
template <> __device__ __forceinline__ void dft_r<16>(float2 (&v)[16])
{
    float2 y[16];
    dft16(v, y);
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = y[q];
}

// The last Stockham pass (sub-transform size 256, radix R = L / 256) of the
// thread's 16 elements x[s] = X[j + T s], T = L / 16: butterfly b = j + T u,
// u < 16 / R, takes X[b + 256 r] = x[u + (16 / R) r], twiddles them by
// w_L^{r b} (W: w_4096^q) and leaves output q at x[u + (16 / R) q], i.e.
// output index j + T s again.
template <int R>
__device__ __forceinline__ void last_pass(float2 (&x)[16], int j, int T, const float2 *__restrict__ W)
{
    constexpr int U = 16 / R;
    const int wst = 4096 / (256 * R);  // w_L^e = w_4096^{e wst}, L = 256 R
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int step = (j + T * u) * wst;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[u + U * r];
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(W + r * step));
        dft_r<R>(v);
#pragma unroll
        for (int q = 0; q < R; ++q) x[u + U * q] = v[q];
    }
}

// An integer the compiler must treat as unknown: keeps the exchange-buffer
// addresses of fft_reg from being hoisted out of the Bluestein loop (they
// would then occupy registers across both transforms).
__device__ __forceinline__ int opaque(int v)
{
    int o;
    asm volatile("mov.b32 %0, %1;" : "=r"(o) : "r"(v));
    return o;
}

// Inverse FFT (sign +, unnormalised) of length L = 16 T of the thread's elements x[s] =
// X[j + T s]; returns them as Y[j + T s].  xb is the map's padded exchange
// region (L + L / 16 elements).  All threads of the CTA call it (it holds
// barriers); inactive threads compute nothing.
__device__ __forceinline__ void fft_reg(float2 (&x)[16], float2 *xb, int j, int T, int L, const float2 *__restrict__ W,
                                        bool active)
{
    float2 y[16];
    j = opaque(j);
    // element j + T r sits at PX(j) + r S, S = T + T / 16 (T is a multiple of 16)
    const int S = opaque(T + (T >> 4));
    const float2 *rd = xb + PX(j);
    // pass 1: sub-transform size 1, radix 16: butterfly j takes X[j + T r]
    if (active) dft16(x, y);
    __syncthreads();  // the exchange buffer's previous contents have been read
    if (active) {
        float2 *wr = xb + 17 * j;  // PX(16 j + q) = 17 j + q
#pragma unroll
        for (int q = 0; q < 16; ++q) wr[q] = y[q];
    }
    __syncthreads();
    // pass 2: sub-transform size 16, radix 16: twiddle w_256^{r (j mod 16)}
    if (active) {
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = rd[r * S];
        const int step = 16 * (j & 15);
#pragma unroll
        for (int r = 1; r < 16; ++r) x[r] = cmul(x[r], __ldg(W + r * step));
        dft16(x, y);
    }
    __syncthreads();
    if (active) {
        float2 *wr = xb + PX((j >> 4) * 256 + (j & 15));  // PX(base + 16 q) = PX(base) + 17 q
#pragma unroll
        for (int q = 0; q < 16; ++q) wr[17 * q] = y[q];
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int q = 0; q < 16; ++q) x[q] = rd[q * S];
        // pass 3: sub-transform size 256, radix L / 256
        switch (L) {
        case 512: last_pass<2>(x, j, T, W); break;
        case 1024: last_pass<4>(x, j, T, W); break;
        case 2048: last_pass<8>(x, j, T, W); break;
        case 4096: last_pass<16>(x, j, T, W); break;
        default: break;  // L = 256: two passes
        }
    }
}

// ------------------------------------------------------------- PTX helpers --
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait (kWaitNs); false if it ran out
__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_try(bar, parity))
        if (gtimer() - t0 > kWaitNs) return false;
    return true;
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

struct RegArgs {
    const float2 *delta;  // [ring][m][map] (per plan) ; many requests: mp.delta[req], [ring][m]
    float *map;
    int nmaps, ngroups, nunits;
    int slot_rows;        // orders per shared-memory slot (a multiple of kBoxRows)
    int use_tma;
    const int2 *items;    // many requests: (request, ring) per unit
    const DevPlan *plans;
    int *status;          // set to SHT_ETIMEOUT when a bounded wait ran out
};

template <bool MULTI>
__global__ void __launch_bounds__(kRT, 2)
ring_reg_kernel(const __grid_constant__ DevPlan P0, const __grid_constant__ RegArgs A,
                const __grid_constant__ CUtensorMap tmap, const __grid_constant__ MultiTcPtrs mp)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    float4 *slot0 = reinterpret_cast<float4 *>(smem);  // 2 slots of slot_rows orders x 2 maps
    float2 *xbuf = reinterpret_cast<float2 *>(smem + (size_t)2 * A.slot_rows * sizeof(float4));
    const int tid = threadIdx.x;
    const float2 *__restrict__ W = P0.w2_32;  // e^{2 pi i q / 4096}

    // unit -> (plan, ring, first map, maps, Delta, map)
    struct Unit {
        const DevPlan *P;
        int r, b0, gn;
        const float2 *delta;
        float *map;
        int nmaps;
    };
    auto unit_of = [&](int u) {
        Unit U;
        if constexpr (MULTI) {
            const int2 it = A.items[u];
            U.P = A.plans + it.x;
            U.r = it.y;
            U.b0 = 0;
            U.gn = 1;
            U.delta = static_cast<const float2 *>(mp.delta[it.x]);
            U.map = static_cast<float *>(mp.map[it.x]);
            U.nmaps = 1;
        } else {
            const int li = u / A.ngroups, g = u - li * A.ngroups;
            U.P = &P0;
            U.r = P0.rf_rings[li];
            U.b0 = 2 * g;
            U.gn = min(2, A.nmaps - 2 * g);
            U.delta = A.delta;
            U.map = A.map;
            U.nmaps = A.nmaps;
        }
        return U;
    };
    // bring unit u's Delta block into slot s (TMA: thread 0; else every thread, one commit group)
    auto issue = [&](int u, int s) {
        float4 *dst = slot0 + (size_t)s * A.slot_rows;
        if (A.use_tma) {
            if (tid == 0 && u < A.nunits) {
                const Unit U = unit_of(u);
                const int M1 = ring_mtop(*U.P, U.r) + 1;  // orders past it are never read
                const int nbox = (M1 + kBoxRows - 1) / kBoxRows;
                SHT_CHECK(U.P->dbg, nbox * kBoxRows <= A.slot_rows && U.b0 % 2 == 0 && U.b0 + 2 <= U.nmaps, 308);
                const uint32_t b = smem_u32(&bar[s]);
                asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(b),
                             "r"((uint32_t)(nbox * kBoxRows * 16))
                             : "memory");
                for (int k = 0; k < nbox; ++k) {
                    asm volatile(
                        "cp.async.bulk.tensor.3d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
                            smem_u32(dst + (size_t)k * kBoxRows)),
                        "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(4 * (U.b0 / 2)), "r"(k * kBoxRows), "r"(U.r), "r"(b)
                        : "memory");
                }
            }
        } else {
            if (u < A.nunits) {
                const Unit U = unit_of(u);
                const int M = U.P->mmax;
                const int Mr = ring_mtop(*U.P, U.r);  // orders past it are never read
                const float2 *src = U.delta + (size_t)U.r * (M + 1) * U.nmaps + U.b0;
                const bool v16 = U.gn == 2 && ((reinterpret_cast<uintptr_t>(src) & 15) == 0) && (U.nmaps % 2 == 0);
                SHT_CHECK(U.P->dbg, M < A.slot_rows, 309);
                for (int m = tid; m <= Mr; m += kRT) {
                    const float2 *sm = src + (size_t)m * U.nmaps;
                    float2 *d = reinterpret_cast<float2 *>(dst + m);
                    if (v16) {
                        cp_async16(d, sm);
                    } else {
                        cp_async8(d, sm);
                        if (U.gn == 2) cp_async8(d + 1, sm + 1);
                    }
                }
            }
            cp_async_commit();
        }
    };

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    issue(blockIdx.x, 0);
    issue(blockIdx.x + gridDim.x, 1);

    for (int i = 0;; ++i) {
        const int u = blockIdx.x + i * gridDim.x;
        if (u >= A.nunits) break;
        const int s = i & 1;
        bool ok = true;
        if (A.use_tma)
            ok = mbar_wait_bounded(smem_u32(&bar[s]), (uint32_t)((i >> 1) & 1));
        else
            cp_async_wait1();
        if (__syncthreads_or(!ok)) {
            // a Delta copy did not arrive in time: record it, give the copies
            // issued into both slots one more bounded wait, and leave (all threads)
            if (tid == 0) {
                atomicExch(A.status, SHT_ETIMEOUT);
                for (int k = 0; k < 2; ++k)
                    if (u + k * (int)gridDim.x < A.nunits)
                        mbar_wait_bounded(smem_u32(&bar[(i + k) & 1]), (uint32_t)(((i + k) >> 1) & 1));
            }
            __syncthreads();
            return;
        }
        const Unit U = unit_of(u);
        const DevPlan &P = *U.P;
        const int r = U.r;
        const int n = P.nphi[r];
        const int M = ring_mtop(P, r);  // Delta_m is zero past it
        const int N = n >> 1;
        const int Lc = P.rf_len[r];
        const bool blue = Lc < 0;
        const int L = blue ? -Lc : Lc;
        const int T = L >> 4;                // threads per map
        const int C = kRT / T;               // maps at once
        const int h = tid / T, j = tid - h * T;
        const int rounds = (U.gn + C - 1) / C;
        const float2 *Tw = P.tw32 + P.twofs[r];  // e^{i pi q / n}, q < 2n
        const int ps = P.ps[r];
        const double phi0 = P.phi0[r];
        const int n2 = 2 * n;
        // phase indices (m ps) mod 2n of the thread's first bin, and their steps
        const int pj = ps >= 0 ? (j * ps) % n2 : 0;
        const int dpk = ps >= 0 ? (T * ps) % n2 : 0;
        const int pN = ps >= 0 ? (N * ps) % n2 : 0;
        const float4 *slot = slot0 + (size_t)s * A.slot_rows;
        float2 *xb = xbuf + (size_t)h * (L + (L >> 4));
        const float2 *chirp = blue ? P.rf_ch32 + P.rf_ch_ofs[r] : nullptr;
        const float2 *bh = blue ? P.rf_bh32 + P.rf_bh_ofs[r] : nullptr;

        for (int rd = 0; rd < rounds; ++rd) {
            const int gi = rd * C + h;
            const bool active = h < C && gi < U.gn;
            if (rd > 0) __syncthreads();  // the previous round's last reads of the exchange buffer
            if (active) {
                const float2 *D = reinterpret_cast<const float2 *>(slot) + gi;  // Delta_m at D[2 m]
                SHT_CHECK(P.dbg, M < A.slot_rows && 2 * N <= n && N <= (blue ? L : L), 301);
                SHT_CHECK(P.dbg, (h + 1) * (L + (L >> 4)) <= kXElems, 302);
                // Table phases (phi0 = pi ps / n): the aliases m = k + t n of bin k share
                // the phase e^{i k phi0} up to sg^t, sg = (-1)^ps, and the conjugated
                // aliases m = t n - k contribute sg^t conj(Delta_m) e^{i k phi0}, so
                //   F_k = e^{i k phi0} A_k,  A_k = sum_t sg^t Delta_{k + t n} + sum_{t >= 1} sg^t conj(Delta_{t n - k}),
                // and with B = A_{N - k}, c = e^{-i N phi0}:
                //   Z_k = e^{i k phi0} ((A + c conj B) + i w^k (A - c conj B)).
                // Arbitrary phi0 (ps < 0): every order gets its own phase.
                const float sg = (ps & 1) ? -1.f : 1.f;
                auto alias_sum = [&](int m1, int m2) {
                    float2 acc = c2(0.f, 0.f);
                    float f = 1.f;
                    for (int m = m1; m <= M; m += n, f *= sg) acc = cadd(acc, c2(f * D[2 * m].x, f * D[2 * m].y));
                    f = sg;
                    for (int m = m2; m <= M; m += n, f *= sg) acc = cadd(acc, c2(f * D[2 * m].x, -f * D[2 * m].y));
                    return acc;
                };
                auto phased_sum = [&](int m1, int m2) {
                    float2 acc = c2(0.f, 0.f);
                    for (int m = m1; m <= M; m += n) {
                        double sn, cs;
                        sincos((double)m * phi0, &sn, &cs);
                        acc = cadd(acc, cmul(D[2 * m], c2((float)cs, (float)sn)));
                    }
                    for (int m = m2; m <= M; m += n) {
                        double sn, cs;
                        sincos((double)m * phi0, &sn, &cs);
                        acc = cadd(acc, cconj(cmul(D[2 * m], c2((float)cs, (float)sn))));
                    }
                    return acc;
                };
                const float2 cN = cconj(__ldg(Tw + pN));  // e^{-i N phi0}
                // rings longer than M: bin k has at most the orders k and n - k
                // (and N - k, N + k for its mirror), no loops
                const bool one_alias = n > M && ps >= 0;
                auto dget = [&](int m) { return m <= M ? D[2 * m] : c2(0.f, 0.f); };
                // the FFT input X[k], k = j + T q, goes to the thread's own slots of the
                // exchange buffer (read back by the same thread: no barrier needed)
                int pk = pj;  // (k ps) mod 2n
#pragma unroll 4
                for (int q = 0; q < 16; ++q) {
                    const int k = j + T * q;
                    float2 z = c2(0.f, 0.f);
                    if (k < N) {
                        const float2 w = __ldg(Tw + SHT_IDX(P.dbg, 2 * k, n2, 305));  // e^{2 pi i k / n}
                        if (one_alias) {
                            const float2 ph = __ldg(Tw + SHT_IDX(P.dbg, pk, n2, 304));  // e^{i k phi0}
                            const float2 d1 = dget(k), d2 = dget(n - k), d3 = dget(N - k), d4 = dget(N + k);
                            const float2 a = c2(d1.x + sg * d2.x, d1.y - sg * d2.y);
                            const float2 b = cmul(cN, c2(d3.x + sg * d4.x, -(d3.y - sg * d4.y)));
                            z = cmul(ph, cadd(cadd(a, b), cmuli(cmul(w, csub(a, b)))));
                        } else if (ps >= 0) {
                            const float2 ph = __ldg(Tw + pk);  // e^{i k phi0}
                            const float2 a = alias_sum(k, n - k);
                            const float2 b = cmul(cN, cconj(alias_sum(N - k, N + k)));
                            z = cmul(ph, cadd(cadd(a, b), cmuli(cmul(w, csub(a, b)))));
                        } else {
                            const float2 f = phased_sum(k, n - k), g = cconj(phased_sum(N - k, N + k));
                            z = cadd(cadd(f, g), cmuli(cmul(w, csub(f, g))));
                        }
                        if (blue) z = cconj(cmul(z, __ldg(chirp + k)));
                    }
                    xb[SHT_IDX(P.dbg, PX(k), L + (L >> 4), 303)] = z;
                    pk += dpk;
                    if (pk >= n2) pk -= n2;
                }
            }
            if (rd == rounds - 1) {
                __syncthreads();  // the slot has been read
                issue(u + 2 * gridDim.x, s);
            }
            float2 x[16];
            if (active) {
#pragma unroll
                for (int q = 0; q < 16; ++q) x[q] = xb[PX(j + T * q)];
            }
            // Bluestein: the forward transform as conj(IFFT(conj(.))) -- the fold
            // stored conj(Z c) -- then the product with the chirp spectrum
#pragma unroll 1
            for (int f = 0; f < (blue ? 2 : 1); ++f) {
                fft_reg(x, xb, j, T, L, W, active);
                if (blue && f == 0 && active) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) x[q] = cmul(cconj(x[q]), __ldg(bh + SHT_IDX(P.dbg, j + T * q, L, 307)));
                }
            }
            if (active) {
                SHT_CHECK(P.dbg, P.ofs[r] + n <= P.npix && U.b0 + gi < U.nmaps, 306);
                float *out = U.map + (size_t)(U.b0 + gi) * P.npix + P.ofs[r];
                const bool al = (reinterpret_cast<uintptr_t>(out) & 7) == 0;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int k = j + T * q;
                    if (k < N) {
                        const float2 v = blue ? cmul(x[q], __ldg(chirp + k)) : x[q];
                        if (al) {
                            reinterpret_cast<float2 *>(out)[k] = v;
                        } else {
                            out[2 * k] = v.x;
                            out[2 * k + 1] = v.y;
                        }
                    }
                }
            }
        }
    }
    if (!A.use_tma) asm volatile("cp.async.wait_all;" ::: "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

size_t reg_smem_bytes(int slot_rows) { return (size_t)2 * slot_rows * sizeof(float4) + (size_t)kXElems * sizeof(float2); }

int slot_rows_for(int mmax) { return ((mmax + 1 + kBoxRows - 1) / kBoxRows) * kBoxRows; }

template <bool MULTI>
cudaError_t launch_reg(const DevPlan &P, const RegArgs &A0, const CUtensorMap &tm, const MultiTcPtrs &mp,
                       cudaStream_t st)
{
    RegArgs A = A0;
    const size_t smem = reg_smem_bytes(A.slot_rows);
    auto k = ring_reg_kernel<MULTI>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kRT, smem)) != cudaSuccess) return e;
    const int grid = std::max(1, std::min(A.nunits, nsm * std::max(1, per)));
    k<<<grid, kRT, smem, st>>>(P, A, tm, mp);
    return cudaGetLastError();
}

}  // namespace

// The driver's tensor-map encoder (nullptr when the driver has none), shared
// with the other kernel files.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn(); }

size_t ring_reg_smem_bytes(int mmax) { return reg_smem_bytes(slot_rows_for(mmax)); }

cudaError_t launch_ring_reg(const DevPlan &P, const float2 *delta_rm, float *map, int nmaps, int *status,
                            cudaStream_t st)
{
    if (nmaps <= 0 || P.rf_n <= 0) return cudaSuccess;
    RegArgs A{};
    A.delta = delta_rm;
    A.map = map;
    A.nmaps = nmaps;
    A.ngroups = (nmaps + 1) / 2;
    A.nunits = P.rf_n * A.ngroups;
    A.slot_rows = slot_rows_for(P.mmax);
    A.status = status;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    A.use_tma = 0;
    auto enc = encode_fn();
    if (enc && nmaps % 2 == 0 && (reinterpret_cast<uintptr_t>(delta_rm) & 15) == 0) {
        // Delta as a 3-D array of floats: (2 nmaps) x (M + 1) x nrings; box 4 floats (2 maps) x 256 orders
        const cuuint64_t dims[3] = {(cuuint64_t)2 * nmaps, (cuuint64_t)P.mmax + 1, (cuuint64_t)P.nrings};
        const cuuint64_t strides[2] = {(cuuint64_t)2 * nmaps * sizeof(float),
                                       (cuuint64_t)2 * nmaps * sizeof(float) * (P.mmax + 1)};
        const cuuint32_t box[3] = {4, (cuuint32_t)kBoxRows, 1};
        const cuuint32_t es[3] = {1, 1, 1};
        const CUresult cr = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2 *>(delta_rm), dims, strides,
                                box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        A.use_tma = cr == CUDA_SUCCESS ? 1 : 0;
    }
    static const MultiTcPtrs none{};
    return launch_reg<false>(P, A, tm, none, st);
}

cudaError_t launch_ring_reg_multi(const DevPlan &P, const DevPlan *plans_dev, const int2 *items, int nitems,
                                  int max_mmax, const MultiTcPtrs &mp, int *status, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    RegArgs A{};
    A.nmaps = 1;
    A.ngroups = 1;
    A.nunits = nitems;
    A.slot_rows = slot_rows_for(max_mmax);
    A.use_tma = 0;
    A.items = items;
    A.plans = plans_dev;
    A.status = status;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    return launch_reg<true>(P, A, tm, mp, st);
}

}  // namespace sht
