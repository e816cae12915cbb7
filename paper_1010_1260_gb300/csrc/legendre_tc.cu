// Legendre step, precision forms: FP64 recurrence, tensor-core contraction.
//
// For each order m the contraction of Eq. DeltaDef is a pair of dense GEMMs
// over the ring pairs r (rows), the degrees l of one parity (the K axis) and
// the maps (columns c = 2 b + {re, im}):
//     E[r, c] = sum_{l - m even} p_l(x_r) B[l, c],  O[r, c] = the same over odd l - m,
//     B[l, c] = C_l a_lm(map b, re/im),   lambda_lm = C_l p_l,
// and Delta_m(north) = E + O, Delta_m(south) = E - O (sec. 2.2.1 symmetry).
// The p_l come from the FP64 recurrence of Eq. assLegRec (scaled form, see
// legendre_fp64.cu), with the exponent tracking of Algorithm 2; they are
// split into TF32 (hi, lo) or BF16 (2 or 3) pieces, B likewise, and the
// products hi*hi + hi*lo + lo*hi (+ the second-order terms for 3 pieces)
// accumulate in FP32 in tensor memory.
//
// CTA (192 threads) = (block of 128 ring pairs, m, group of <= 64 maps):
//   warps 0-3  one ring pair per thread: FP64 recurrence -> split pieces ->
//              swizzled K-major A tiles in shared memory; at the end, the
//              epilogue reads E and O from tensor memory (tcgen05.ld) and
//              writes Delta in FP32;
//   warp 4     allocates tensor memory and loads the B tiles with TMA;
//   warp 5     one thread issues tcgen05.mma (M = 128, N = 2 x maps, K = one
//              chunk) and releases stages with tcgen05.commit.
// Stages hold KC degrees of each parity (one MMA K step); NS stages rotate
// through mbarriers.  Every wait is bounded by a global-timer limit; on
// timeout the CTA records an error in the plan's status word, drains its
// copies and MMAs (again bounded), frees its tensor memory and returns.
#include "sht.h"
#include "sht_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

namespace sht {
namespace {

constexpr uint64_t kTimeoutNs = 2000000000ull;  // 2 s per wait
constexpr int kRows = 128;                      // ring pairs per CTA = MMA M
constexpr int kThreads = 192;
constexpr int kRowBytes = 32;                   // one K chunk per tile row (SW32 swizzle)
constexpr int kTileBytes = kRows * kRowBytes;   // 4 KB per operand tile (N <= 128 rows for B)

// ------------------------------------------------------------- PTX helpers --

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the given phase parity.  Returns false (and raises the
// CTA's abort flag) after kTimeoutNs, or at once if another role aborted.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > kTimeoutNs) {
            *abort_flag = 1;
            return false;
        }
    }
}
// Bounded wait used while draining after an abort (does not look at the flag).
__device__ bool mbar_drain(uint32_t bar, uint32_t parity)
{
    const uint64_t t0 = gtimer();
    while (!mbar_try_wait(bar, parity)) {
        if (gtimer() - t0 > kTimeoutNs) return false;
    }
    return true;
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
template <bool BF16>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    if (BF16) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// K-major operand tile with the 32-byte swizzle: rows of 32 bytes, 8-row
// groups 256 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw32(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(256u >> 4) << 32;        // stride byte offset: 8 rows x 32 bytes
    d |= (uint64_t)1 << 46;                  // descriptor version
    d |= (uint64_t)6 << 61;                  // layout: 32-byte swizzle
    return d;
}
// Instruction descriptor: FP32 accumulator, K-major A and B, M = 128.
template <bool BF16>
__host__ __device__ constexpr uint32_t idesc(int n)
{
    return (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kRows >> 4) << 24);
}

// FP64 -> FP32 rounded to nearest (ties away from zero) on the integer pipe,
// so the conversion costs no FP64 issue slot.  Values below the FP32 normal
// range become 0; |p| is bounded far below the FP32 maximum.
__device__ __forceinline__ float rn_f32(double d)
{
    const int hi = __double2hiint(d);
    const unsigned lo = (unsigned)__double2loint(d);
    const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
    const unsigned sign = (unsigned)hi & 0x80000000u;
    const unsigned man = (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rbit = (lo >> 28) & 1u;  // first dropped mantissa bit
    const unsigned bits = (e <= 0) ? sign : (sign | ((((unsigned)e << 23) | man) + rbit));
    return __uint_as_float(bits);
}
__device__ __forceinline__ uint32_t rn_tf32_bits(float f)
{
    return (__float_as_uint(f) + 0x1000u) & 0xFFFFE000u;
}
__device__ __forceinline__ uint32_t rn_bf16_bits(float f)
{
    return (__float_as_uint(f) + 0x8000u) & 0xFFFF0000u;
}

// Split v into NP pieces; TF32: fp32 bit patterns; BF16: upper 16 bits used.
template <bool BF16, int NP>
__device__ __forceinline__ void split_pieces(float v, uint32_t (&out)[NP])
{
    float r = v;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const uint32_t b = BF16 ? rn_bf16_bits(r) : rn_tf32_bits(r);
        out[i] = b;
        r = r - __uint_as_float(b);
    }
}

__device__ __forceinline__ bool above_hi(double v)
{
    const int e = (__double2hiint(v) >> 20) & 0x7ff;
    return e > 1023 + kScaleHi;
}

// tensor-memory columns for the E and O accumulators (power of two >= 32)
__device__ __forceinline__ uint32_t tmem_cols(int ncols)
{
    const int need = 2 * ncols;
    return need <= 32 ? 32u : (need <= 64 ? 64u : (need <= 128 ? 128u : 256u));
}

template <bool BF16, int NPA, int NPB>
struct Cfg {
    static constexpr int KC = BF16 ? 16 : 8;   // degrees of one parity per stage = MMA K
    static constexpr int VEC = BF16 ? 8 : 4;   // values per 16-byte chunk
    static constexpr int NCHUNK = KC / VEC;    // 16-byte chunks per tile row (= 2)
    static constexpr int A_TILES = 2 * NPA;    // [parity][piece]
    static constexpr int B_TILES = 2 * NPB;
    static constexpr int STAGE_BYTES = (A_TILES + B_TILES) * kTileBytes;
    static constexpr int NS = (STAGE_BYTES * 3 <= 100 * 1024) ? 3 : 2;
    static constexpr int NPROD = (NPA == 2 && NPB == 2) ? 3 : 6;
    static constexpr int SMEM = NS * STAGE_BYTES + 1024 /* align */ + 256 /* barriers */;
};

template <int NPA, int NPB>
__device__ __forceinline__ void product_pieces(int i, int &ia, int &ib)
{
    // (0,0) (0,1) (1,0) then (0,2) (1,1) (2,0)
    const int a[6] = {0, 0, 1, 0, 1, 2};
    const int b[6] = {0, 1, 0, 2, 1, 0};
    ia = a[i];
    ib = b[i];
}

template <bool BF16, int NPA, int NPB>
__global__ void __launch_bounds__(kThreads, 2)
legendre_tc_kernel(const DevPlan P, const __grid_constant__ CUtensorMap tmB, const int *__restrict__ seg_off,
                   float2 *__restrict__ delta, int nmaps, int ncols, int *__restrict__ status)
{
    using C = Cfg<BF16, NPA, NPB>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned stage area
    const uint32_t base_u32 = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (base_u32 & 1023u)) & 1023u;
    unsigned char *stage0 = smem_raw + pad;
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage0 + C::NS * C::STAGE_BYTES);
    // bars: full_a[NS], full_b[NS], empty[NS], acc_full
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int m = blockIdx.y;
    const int L = P.lmax;
    const int pair_base = blockIdx.x * kRows;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nstages = (L - m + 1 + 2 * C::KC - 1) / (2 * C::KC);

    auto bar_full_a = [&](int s) { return smem_u32(&bars[s]); };
    auto bar_full_b = [&](int s) { return smem_u32(&bars[C::NS + s]); };
    auto bar_empty = [&](int s) { return smem_u32(&bars[2 * C::NS + s]); };
    const uint32_t bar_acc = smem_u32(&bars[3 * C::NS]);
    auto a_tile = [&](int s, int par, int piece) {
        return stage0 + s * C::STAGE_BYTES + (par * NPA + piece) * kTileBytes;
    };
    auto b_tile = [&](int s, int par, int piece) {
        return stage0 + s * C::STAGE_BYTES + (C::A_TILES + par * NPB + piece) * kTileBytes;
    };

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < C::NS; ++s) {
            mbar_init(bar_full_a(s), 4);
            mbar_init(bar_full_b(s), 1);
            mbar_init(bar_empty(s), 1);
        }
        mbar_init(bar_acc, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        // tensor memory: E in columns [0, ncols), O in [ncols, 2 ncols)
        const uint32_t cols = tmem_cols(ncols);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp < 4) {
        // ------------------------------------------------------ producers --
        const int t = threadIdx.x;  // row = ring pair within the block
        const int pair = pair_base + t;
        const bool live = pair < P.npairs;
        double x = 0.0, p0 = 0.0, p1 = 0.0;
        int k = 0;
        if (live) {
            x = P.pair_x[pair];
            p1 = P.start_v[(size_t)m * P.npairs + pair];
            k = P.start_k[(size_t)m * P.npairs + pair];
        }
        const long long mofs = (long long)m * (2 * L + 3 - m) / 2;
        // swizzled byte offset of row t, chunk c inside a tile
        auto chunk_off = [&](int c) { return t * kRowBytes + ((c ^ ((t >> 2) & 1)) << 4); };
        int l = m;
        bool ok = true;
        for (int i = 0; i < nstages && ok; ++i) {
            const int s = i % C::NS;
            const uint32_t ph = (uint32_t)(i / C::NS) & 1u;
            ok = mbar_wait(bar_empty(s), ph ^ 1u, &s_abort);
            if (!ok) break;
#pragma unroll
            for (int c = 0; c < C::NCHUNK; ++c) {
                uint32_t pe[NPA][C::VEC], po[NPA][C::VEC];
#pragma unroll
                for (int v = 0; v < C::VEC; ++v) {
#pragma unroll
                    for (int par = 0; par < 2; ++par) {
                        const double val = (k == 0 && l <= L) ? p1 : 0.0;
                        uint32_t pc[NPA];
                        split_pieces<BF16, NPA>(rn_f32(val), pc);
#pragma unroll
                        for (int q = 0; q < NPA; ++q) {
                            if (par == 0) pe[q][v] = pc[q];
                            else po[q][v] = pc[q];
                        }
                        // advance to l + 1
                        const double A = (l + 1 <= L) ? __ldg(&P.coefA[mofs + (l + 1 - m)]) : 0.0;
                        const double tt = fma(A * x, p1, -p0);
                        p0 = p1;
                        p1 = tt;
                        if (k < 0 && above_hi(p1)) {
                            p1 *= 0x1p-512;
                            p0 *= 0x1p-512;
                            k += 1;
                        }
                        ++l;
                    }
                }
#pragma unroll
                for (int q = 0; q < NPA; ++q) {
                    uint4 we, wo;
                    if (BF16) {
                        we = make_uint4((pe[q][0] >> 16) | (pe[q][1] & 0xFFFF0000u),
                                        (pe[q][2] >> 16) | (pe[q][3] & 0xFFFF0000u),
                                        (pe[q][4 % C::VEC] >> 16) | (pe[q][5 % C::VEC] & 0xFFFF0000u),
                                        (pe[q][6 % C::VEC] >> 16) | (pe[q][7 % C::VEC] & 0xFFFF0000u));
                        wo = make_uint4((po[q][0] >> 16) | (po[q][1] & 0xFFFF0000u),
                                        (po[q][2] >> 16) | (po[q][3] & 0xFFFF0000u),
                                        (po[q][4 % C::VEC] >> 16) | (po[q][5 % C::VEC] & 0xFFFF0000u),
                                        (po[q][6 % C::VEC] >> 16) | (po[q][7 % C::VEC] & 0xFFFF0000u));
                    } else {
                        we = make_uint4(pe[q][0], pe[q][1], pe[q][2 % C::VEC], pe[q][3 % C::VEC]);
                        wo = make_uint4(po[q][0], po[q][1], po[q][2 % C::VEC], po[q][3 % C::VEC]);
                    }
                    *reinterpret_cast<uint4 *>(a_tile(s, 0, q) + chunk_off(c)) = we;
                    *reinterpret_cast<uint4 *>(a_tile(s, 1, q) + chunk_off(c)) = wo;
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_full_a(s));
        }
        // ------------------------------------------------------- epilogue --
        if (ok) ok = mbar_wait(bar_acc, 0u, &s_abort);
        if (ok) {
            tc_fence_after();
            const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
            const int2 rr = live ? P.pair_ring[pair] : make_int2(0, -1);
            const int M1 = P.mmax + 1;
            for (int c0 = 0; c0 < ncols; c0 += 32) {
                uint32_t ev[32], ov[32];
                tmem_ld32(tmem + lane_base + (uint32_t)c0, ev);
                tmem_ld32(tmem + lane_base + (uint32_t)(ncols + c0), ov);
                if (live) {
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        const int b = (c0 + j) >> 1;
                        if (b < nmaps) {
                            const float er = __uint_as_float(ev[j]), ei = __uint_as_float(ev[j + 1]);
                            const float orr = __uint_as_float(ov[j]), oi = __uint_as_float(ov[j + 1]);
                            float2 *d = delta + (size_t)b * P.nrings * M1;
                            d[(size_t)rr.x * M1 + m] = make_float2(er + orr, (m == 0) ? 0.f : ei + oi);
                            if (rr.y >= 0)
                                d[(size_t)rr.y * M1 + m] = make_float2(er - orr, (m == 0) ? 0.f : ei - oi);
                        }
                    }
                }
            }
        }
    } else if (warp == 4) {
        // ------------------------------------------------------ TMA loads --
        int issued = 0;
        if (lane == 0) {
            const int off0 = seg_off[2 * m], off1 = seg_off[2 * m + 1];
            const uint32_t bytes = (uint32_t)(2 * NPB * ncols * kRowBytes);
            for (int i = 0; i < nstages; ++i) {
                const int s = i % C::NS;
                const uint32_t ph = (uint32_t)(i / C::NS) & 1u;
                if (!mbar_wait(bar_empty(s), ph ^ 1u, &s_abort)) break;
                mbar_expect_tx(bar_full_b(s), bytes);
#pragma unroll
                for (int q = 0; q < NPB; ++q) {
                    tma_load_2d(smem_u32(b_tile(s, 0, q)), &tmB, off0 + i * C::KC, q * ncols, bar_full_b(s));
                    tma_load_2d(smem_u32(b_tile(s, 1, q)), &tmB, off1 + i * C::KC, q * ncols, bar_full_b(s));
                }
                ++issued;
            }
            // after an abort, let the copies in flight land before the CTA exits
            if (s_abort) {
                for (int i = (issued > C::NS ? issued - C::NS : 0); i < issued; ++i) {
                    const int s = i % C::NS;
                    mbar_drain(bar_full_b(s), (uint32_t)(i / C::NS) & 1u);
                }
            }
        }
    } else {
        // ----------------------------------------------------------- MMA --
        if (lane == 0) {
            const uint32_t id = idesc<BF16>(ncols);
            int done = 0;
            for (int i = 0; i < nstages; ++i) {
                const int s = i % C::NS;
                const uint32_t ph = (uint32_t)(i / C::NS) & 1u;
                if (!mbar_wait(bar_full_a(s), ph, &s_abort)) break;
                if (!mbar_wait(bar_full_b(s), ph, &s_abort)) break;
                tc_fence_after();
#pragma unroll
                for (int par = 0; par < 2; ++par) {
                    const uint32_t d = tmem + (uint32_t)(par * ncols);
#pragma unroll
                    for (int pr = 0; pr < C::NPROD; ++pr) {
                        int ia, ib;
                        product_pieces<NPA, NPB>(pr, ia, ib);
                        const uint64_t ad = sdesc_sw32(smem_u32(a_tile(s, par, ia)));
                        const uint64_t bd = sdesc_sw32(smem_u32(b_tile(s, par, ib)));
                        tc_mma<BF16>(d, ad, bd, id, (i > 0 || pr > 0) ? 1u : 0u);
                    }
                }
                tc_commit(bar_empty(s));
                ++done;
            }
            if (done == nstages) tc_commit(bar_acc);
            else if (done > 0) {
                // drain: the last commit releases its stage once all earlier MMAs finished
                const int i = done - 1;
                mbar_drain(bar_empty(i % C::NS), (uint32_t)(i / C::NS) & 1u);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        const uint32_t cols = tmem_cols(ncols);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
    }
    if (threadIdx.x == 0 && s_abort) atomicExch(status, SHT_ETIMEOUT);
}

// ------------------------------------------------------------ operand prep --
// B[c][seg(m, par) + k] = pieces of C_l a_lm(map c/2, re or im), l = m + par + 2k,
// zero for l > lmax, for maps beyond nmaps and for Im of m = 0.
template <bool BF16, int NPB>
__global__ void prep_b_kernel(const DevPlan P, const double2 *__restrict__ alm, const int *__restrict__ seg_off,
                              void *__restrict__ bout, long long kall, int nmaps, int ncols, int kc)
{
    const int m = blockIdx.y;
    const int L = P.lmax;
    const int nst = (L - m + 1 + 2 * kc - 1) / (2 * kc);
    const int kpad = nst * kc;
    const long long mofs = (long long)m * (2 * L + 3 - m) / 2;
    const int total = 2 * kpad * ncols;  // (par, c, k)
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int k = idx % kpad;
        const int c = (idx / kpad) % ncols;
        const int par = idx / (kpad * ncols);
        const int l = m + par + 2 * k;
        const int b = c >> 1;
        float v = 0.f;
        if (l <= L && b < nmaps && !(m == 0 && (c & 1))) {
            const double2 a = alm[(size_t)b * P.nalm + mofs + (l - m)];
            v = rn_f32(P.coefC[mofs + (l - m)] * ((c & 1) ? a.y : a.x));
        }
        uint32_t pc[NPB];
        split_pieces<BF16, NPB>(v, pc);
        const long long col = seg_off[2 * m + par] + k;
#pragma unroll
        for (int q = 0; q < NPB; ++q) {
            const long long row = (long long)q * ncols + c;
            if (BF16)
                reinterpret_cast<uint16_t *>(bout)[row * kall + col] = (uint16_t)(pc[q] >> 16);
            else
                reinterpret_cast<uint32_t *>(bout)[row * kall + col] = pc[q];
        }
    }
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
    });
    return fn;
}

template <bool BF16, int NPA, int NPB>
cudaError_t run_prep(const DevPlan &P, const TcWork &W, const double2 *alm, int nmaps, cudaStream_t st)
{
    using C = Cfg<BF16, NPA, NPB>;
    const int ncols = tc_ncols(nmaps);
    const int *seg = BF16 ? W.seg_bf16 : W.seg_tf32;
    const long long kall = BF16 ? W.kall_bf16 : W.kall_tf32;
    dim3 grid(64, P.mmax + 1);
    prep_b_kernel<BF16, NPB><<<grid, 256, 0, st>>>(P, alm, seg, W.bbuf, kall, nmaps, ncols, C::KC);
    return cudaGetLastError();
}

template <bool BF16, int NPA, int NPB>
cudaError_t run_main(const DevPlan &P, const TcWork &W, float2 *delta, int nmaps, cudaStream_t st)
{
    using C = Cfg<BF16, NPA, NPB>;
    const int ncols = tc_ncols(nmaps);
    const int *seg = BF16 ? W.seg_bf16 : W.seg_tf32;
    const long long kall = BF16 ? W.kall_bf16 : W.kall_tf32;
    // tensor map over the B pieces: rows (piece, c), columns K
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap tm;
    const cuuint64_t dims[2] = {(cuuint64_t)kall, (cuuint64_t)(NPB * ncols)};
    const cuuint64_t strides[1] = {(cuuint64_t)kall * (BF16 ? 2 : 4)};
    const cuuint32_t box[2] = {(cuuint32_t)C::KC, (cuuint32_t)ncols};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&tm, BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, W.bbuf, dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    auto kern = legendre_tc_kernel<BF16, NPA, NPB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((P.npairs + kRows - 1) / kRows, P.mmax + 1);
    kern<<<grid, kThreads, C::SMEM, st>>>(P, tm, seg, delta, nmaps, ncols, W.status);
    return cudaGetLastError();
}

}  // namespace

size_t tc_bbuf_bytes(const TcWork &W, int prec)
{
    // pieces x 128 columns (the widest launch group) x K
    if (prec == SHT_FP32_TC) return (size_t)2 * 128 * W.kall_tf32 * 4;
    if (prec == SHT_BF16X3_TC) return (size_t)2 * 128 * W.kall_bf16 * 2;
    return (size_t)3 * 128 * W.kall_bf16 * 2;
}

cudaError_t launch_tc_prep(const DevPlan &P, const TcWork &W, int prec, const double2 *alm, int nmaps, cudaStream_t st)
{
    if (nmaps <= 0) return cudaSuccess;
    if (nmaps > kTcMaxMaps) return cudaErrorInvalidValue;
    if (prec == SHT_FP32_TC) return run_prep<false, 2, 2>(P, W, alm, nmaps, st);
    if (prec == SHT_BF16X3_TC) return run_prep<true, 2, 2>(P, W, alm, nmaps, st);
    return run_prep<true, 3, 3>(P, W, alm, nmaps, st);
}

cudaError_t launch_tc_main(const DevPlan &P, const TcWork &W, int prec, float2 *delta, int nmaps, cudaStream_t st)
{
    if (nmaps <= 0) return cudaSuccess;
    if (nmaps > kTcMaxMaps) return cudaErrorInvalidValue;
    if (prec == SHT_FP32_TC) return run_main<false, 2, 2>(P, W, delta, nmaps, st);
    if (prec == SHT_BF16X3_TC) return run_main<true, 2, 2>(P, W, delta, nmaps, st);
    return run_main<true, 3, 3>(P, W, delta, nmaps, st);
}

}  // namespace sht
