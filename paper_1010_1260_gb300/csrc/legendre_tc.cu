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
// Persistent kernel, one CTA (10 warps) per SM; work item = (m, block of 128
// ring pairs) for a group of <= 64 maps, heavy (small m) items first:
//   warps 0-3  one ring pair per thread: FP64 recurrence (recurrence
//              coefficients prefetched a stage ahead and broadcast by warp
//              shuffle, so the only dependent chain is one DFMA per degree)
//              -> pieces -> swizzled K-major A tiles in shared memory;
//   warp 8     allocates tensor memory and loads each stage's B tiles with
//              one bulk copy (the operand prep writes them pre-swizzled and
//              contiguous), prefetching the next stages into L2;
//   warp 9     one thread issues tcgen05.mma (M = 128, N = 2 x maps, K = one
//              chunk) and releases stages with tcgen05.commit;
//   warps 4-7  drain: the MMAs of every 64 degrees accumulate into tensor-
//              memory columns 0-255; the drain warps read the finished group
//              (tcgen05.ld), add it in FP32 (round to nearest) into the item's
//              totals in columns 256-511 (tcgen05.st), release the
//              accumulator, and at the end of an item write Delta through a
//              small shared-memory staging buffer.  Keeping the totals out of
//              shared memory leaves it to the stage ring (4 or 6 stages) and
//              takes the drain's traffic off the producers' shared-memory
//              path.  The tensor core's FP32
//              accumulation rounds toward zero, which over ~400 accumulating
//              MMAs biases the result by ~1e-5; summing short groups on the
//              CUDA cores removes the bias.
// Stages hold KC degrees of each parity (one MMA K step); NS stages rotate
// through mbarriers.  Every wait is bounded by a global-timer limit; on
// timeout the CTA records an error in the plan's status word, drains its
// copies and MMAs (again bounded), frees its tensor memory and returns.
// withhold >= 0 (a test hook, sht_debug_withhold_stage) makes CTA 0 skip the
// copies of its stage number `withhold`, so that the MMA warp's wait for that
// stage runs out: nothing faults, the CTA takes the abort path above.
#include "sht.h"
#include "sht_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <cstdint>
#include <mutex>

namespace sht {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();  // ring_reg.cu
namespace {

constexpr uint64_t kTimeoutNs = 2000000000ull;  // 2 s per wait
constexpr int kRows = 128;                      // ring pairs per CTA = MMA M
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
// Contiguous bulk copy global -> shared completing on an mbarrier, and an L2
// prefetch of a contiguous range (no shared memory used).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(src)), "r"(bytes)
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
// The same load without the wait (tmem_wait_ld before the registers are read).
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 32 consecutive columns of the warp's 32 lanes from registers; tmem_wait_st
// before the registers are reused or the columns are read back.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
        "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
        "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

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
// range become 0; |p| is bounded far below the FP32 maximum.  Bits 29..60 of
// the double are its 9 low exponent bits and the 23 kept mantissa bits: adding
// 2^30 rebiases the exponent by -896 modulo 2^9, which is exact for every FP32
// normal exponent, and the first dropped bit rounds (a carry into the exponent
// is the correct result).
__device__ __forceinline__ float rn_f32(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d);
    const unsigned lo = (unsigned)__double2loint(d);
    const unsigned bits = (__funnelshift_r(lo, hi, 29) + 0x40000000u + ((lo >> 28) & 1u)) | (hi & 0x80000000u);
    return __uint_as_float((hi & 0x7ff00000u) <= 0x38000000u ? (hi & 0x80000000u) : bits);
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

// The coefficient product A_l x of the recurrence, correctly rounded like a
// DMUL but computed on the integer pipes: the FP64 pipe of this part issues two
// instructions per clock per SM, and a recurrence step otherwise spends two of
// them (the product and the FMA).  x is fixed per ring: XInt holds its
// significand shifted to the top of 64 bits (0 for x = 0) and the additive
// exponent/sign term; A is >= 0, normal or zero, and the product is normal.
struct XInt {
    unsigned long long m;    // (1.f_x) 2^63, or 0 when x == 0
    unsigned long long add;  // ((e_x - 1024) << 52) + sign(x) 2^63, modulo 2^64
};
__device__ __forceinline__ XInt xint_of(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    XInt r;
    r.m = ((b << 1) == 0) ? 0ull : ((b << 11) | 0x8000000000000000ull);
    r.add = ((unsigned long long)((long long)((int)((b >> 52) & 0x7ff) - 1024)) << 52) + (b & 0x8000000000000000ull);
    return r;
}
__device__ __forceinline__ double mul_coef(double a, const XInt &X)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const unsigned long long ma = (b << 11) | 0x8000000000000000ull;
    const unsigned long long hi = __umul64hi(ma, X.m);  // (1.f_a)(1.f_x) 2^62, in [2^62, 2^64)
    const unsigned top = (unsigned)(hi >> 63);
    const unsigned sh = 10u + top;                       // 53 significant bits above bit sh
    // round to nearest even: the low product only decides exact halves, so it
    // is folded into bit 0 (strictly below the rounding bit) as a sticky bit
    unsigned long long hs = hi | (unsigned long long)((ma * X.m) != 0ull);
    hs += (unsigned long long)((512u << top) - 1u) + ((hs >> sh) & 1ull);
    const unsigned long long m53 = hs >> sh;  // hidden bit at 2^52 (2^53 after a carry)
    const unsigned long long r = (b & 0x7ff0000000000000ull) + X.add + ((unsigned long long)top << 52) + m53;
    return (b == 0ull || X.m == 0ull) ? 0.0 : __longlong_as_double((long long)r);
}
// degrees (by position in the stage) whose coefficient product runs on the
// integer pipes; the rest are DMULs (as an FMA with +0): both give the same bits
// (bit q of the pattern, q = position of the degree in the stage).  Two of
// every three (q mod 3 != 1): measured at nside 1024, lmax 2048, 64 maps,
// 13.15 ms, against 13.30 and 13.52 for the other two phases of two in three,
// 13.19 for five in seven, 13.34 for seven in ten, 13.59 for one in two, 13.68
// for three in five, 13.89 for three in four and 14.42 for three in eight.
#ifndef SHT_INT_PRODUCT_BITS
#define SHT_INT_PRODUCT_BITS 0x6DB6DB6Du
#endif
__host__ __device__ constexpr bool int_product(int q) { return ((SHT_INT_PRODUCT_BITS >> (q & 31)) & 1u) != 0u; }
template <int Q>
__device__ __forceinline__ double coef_x(double a, double x, const XInt &X)
{
    if constexpr (int_product(Q)) return mul_coef(a, X);
    else return fma(a, x, 0.0);
}

// BF16 pieces of two values at once, as the packed words the A tiles hold (a
// in the low half, b in the high half): cvt.rn.bf16x2.f32 rounds and packs
// both in one instruction off the integer pipes; the residuals are exact.
#ifndef SHT_F2FP_SPLIT
#define SHT_F2FP_SPLIT 1
#endif
template <int NP>
__device__ __forceinline__ void split_pair_bf16(float a, float b, uint32_t (&w)[NP])
{
#pragma unroll
    for (int i = 0; i < NP; ++i) {
#if SHT_F2FP_SPLIT
        uint32_t p;
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p) : "f"(b), "f"(a));
#else
        const uint32_t p = (rn_bf16_bits(a) >> 16) | rn_bf16_bits(b);
#endif
        w[i] = p;
        if (i + 1 < NP) {
            a -= __uint_as_float(p << 16);
            b -= __uint_as_float(p & 0xFFFF0000u);
        }
    }
}

__device__ __forceinline__ bool above_hi(double v)
{
    const int e = (__double2hiint(v) >> 20) & 0x7ff;
    return e > 1023 + kScaleHi;
}

template <bool BF16, int NPA, int NPB>
struct Cfg {
    static constexpr int KC = BF16 ? 16 : 8;   // degrees of one parity per stage = MMA K
    static constexpr int VEC = BF16 ? 8 : 4;   // values per 16-byte chunk
    static constexpr int NCHUNK = KC / VEC;    // 16-byte chunks per tile row (= 2)
    static constexpr int STEPS = 2 * KC;       // consecutive degrees per stage
    static constexpr int A_TILES = 2 * NPA;    // [parity][piece]
    static constexpr int B_TILES = 2 * NPB;
    static constexpr int STAGE_BYTES = (A_TILES + B_TILES) * kTileBytes;
    static constexpr int NPROD = (NPA == 2 && NPB == 2) ? 3 : 6;
    static constexpr int GROUP = 64 / STEPS;   // stages per accumulation group (64 degrees)
    static constexpr int STG_BYTES = 4 * 32 * 16 * 8;  // Delta staging, per drain warp 32 rows x 16 float2
    // stage ring: as deep as shared memory allows (4 of 48 KB, 6 of 32 KB)
    static constexpr int NS = (227 * 1024 - 1024 - 256 - STG_BYTES) / STAGE_BYTES;
    static constexpr int SMEM = NS * STAGE_BYTES + STG_BYTES + 1024 /* align */ + 256 /* barriers */;
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

template <int NPA>
__device__ __forceinline__ void store_words(unsigned char *sbase, int t, int c, const uint32_t (&we)[NPA][4],
                                            const uint32_t (&wo)[NPA][4])
{
    const int off = t * kRowBytes + ((c ^ ((t >> 2) & 1)) << 4);
#pragma unroll
    for (int i = 0; i < NPA; ++i) {
        *reinterpret_cast<uint4 *>(sbase + (0 * NPA + i) * kTileBytes + off) = make_uint4(we[i][0], we[i][1], we[i][2], we[i][3]);
        *reinterpret_cast<uint4 *>(sbase + (1 * NPA + i) * kTileBytes + off) = make_uint4(wo[i][0], wo[i][1], wo[i][2], wo[i][3]);
    }
}

// Store the packed pieces of one 16-byte chunk (VEC values per parity).
template <bool BF16, int NPA, int VEC>
__device__ __forceinline__ void store_chunk(unsigned char *sbase, int t, int c, const uint32_t (&pe)[NPA][VEC],
                                            const uint32_t (&po)[NPA][VEC])
{
    const int off = t * kRowBytes + ((c ^ ((t >> 2) & 1)) << 4);
#pragma unroll
    for (int i = 0; i < NPA; ++i) {
        uint4 we, wo;
        if (BF16) {
            we = make_uint4((pe[i][0] >> 16) | (pe[i][1] & 0xFFFF0000u), (pe[i][2] >> 16) | (pe[i][3] & 0xFFFF0000u),
                            (pe[i][4 % VEC] >> 16) | (pe[i][5 % VEC] & 0xFFFF0000u),
                            (pe[i][6 % VEC] >> 16) | (pe[i][7 % VEC] & 0xFFFF0000u));
            wo = make_uint4((po[i][0] >> 16) | (po[i][1] & 0xFFFF0000u), (po[i][2] >> 16) | (po[i][3] & 0xFFFF0000u),
                            (po[i][4 % VEC] >> 16) | (po[i][5 % VEC] & 0xFFFF0000u),
                            (po[i][6 % VEC] >> 16) | (po[i][7 % VEC] & 0xFFFF0000u));
        } else {
            we = make_uint4(pe[i][0], pe[i][1], pe[i][2 % VEC], pe[i][3 % VEC]);
            wo = make_uint4(po[i][0], po[i][1], po[i][2 % VEC], po[i][3 % VEC]);
        }
        *reinterpret_cast<uint4 *>(sbase + (0 * NPA + i) * kTileBytes + off) = we;
        *reinterpret_cast<uint4 *>(sbase + (1 * NPA + i) * kTileBytes + off) = wo;
    }
}

// One producer stage: 2 KC consecutive degrees of one ring pair (row t),
// written as NPA pieces into the stage's A tiles ([parity][piece], 4 KB
// each, K-major rows of 32 bytes with the 32-byte swizzle).  a_cur holds
// A_{l+1} for the stage's degrees, one per lane.
// The products A_{l+1} x are correctly rounded either way: degrees selected by
// int_product() take them on the integer pipes (mul_coef), the others as
// fma(A, x, +0.0), a DFMA (the FP64 pipe takes a DMUL per 76 cycles and a DFMA
// per 64 per warp), so the FP64 pipe carries 1.33 instead of 2 instructions per
// degree.  BF16 pieces are rounded and packed in pairs (split_pair_bf16).
// SLOW = false (no ring of the warp still rescaled): software-pipelined for
// one warp per SM sub-partition issuing in order -- each degree issues its
// DFMA (the only dependent chain), the product of the degree two ahead, the shuffle of the
// coefficient three ahead, then the integer / FP32 conversion of the current
// value, so the conversions hide under the FP64 work instead of following it.
// SLOW = true: rescaled rings contribute zeros and the rescale test runs once
// per chunk of 2 VEC degrees (the values grow by far less than 2^512 over a chunk).
template <bool BF16, int NPA, bool SLOW>
__device__ __forceinline__ void produce_stage(unsigned char *sbase, int t, double x, const XInt &X, double a_cur, int l,
                                              int L, double &p0, double &p1, int &k)
{
    constexpr int KC = BF16 ? 16 : 8;
    constexpr int VEC = BF16 ? 8 : 4;
    constexpr int NCH = KC / VEC;
    constexpr int STEPS = 2 * KC;
    if constexpr (!SLOW) {
        // A_{l+1} x two degrees ahead, A_{l+1} three degrees ahead: the DFMA of
        // a degree never waits for its DMUL, nor the DMUL for its shuffle.
        double ax0 = coef_x<0>(__shfl_sync(0xffffffffu, a_cur, 0), x, X);
        double ax1 = coef_x<1>(__shfl_sync(0xffffffffu, a_cur, 1), x, X);
        double an = __shfl_sync(0xffffffffu, a_cur, 2);
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            uint32_t pe[NPA][VEC], po[NPA][VEC];
            uint32_t we[NPA][4], wo[NPA][4];  // BF16: packed pairs
#pragma unroll
            for (int vv = 0; vv < VEC; vv += 2) {
                // four degrees (two even, two odd l - m), then the four
                // conversions: independent integer/FP32 chains that the
                // scheduler interleaves under the FP64 latency
                double val[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = c * 2 * VEC + 2 * vv + u;
                    val[u] = p1;
                    const double tt = fma(ax0, p1, -p0);
                    ax0 = ax1;
                    if (q + 2 < STEPS) ax1 = int_product(q + 2) ? mul_coef(an, X) : fma(an, x, 0.0);
                    if (q + 3 < STEPS) an = __shfl_sync(0xffffffffu, a_cur, q + 3);
                    p0 = p1;
                    p1 = tt;
                }
                // degrees past L keep their (finite) values: the B operand's
                // rows there are zero
                float f[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) f[u] = rn_f32(val[u]);
                if constexpr (BF16) {
                    uint32_t e2[NPA], o2[NPA];
                    split_pair_bf16<NPA>(f[0], f[2], e2);
                    split_pair_bf16<NPA>(f[1], f[3], o2);
#pragma unroll
                    for (int i = 0; i < NPA; ++i) {
                        we[i][vv / 2] = e2[i];
                        wo[i][vv / 2] = o2[i];
                    }
                } else {
                    uint32_t cv[4][NPA];
#pragma unroll
                    for (int u = 0; u < 4; ++u) split_pieces<BF16, NPA>(f[u], cv[u]);
#pragma unroll
                    for (int i = 0; i < NPA; ++i) {
                        pe[i][vv] = cv[0][i];
                        po[i][vv] = cv[1][i];
                        pe[i][vv + 1] = cv[2][i];
                        po[i][vv + 1] = cv[3][i];
                    }
                }
            }
            if constexpr (BF16) store_words<NPA>(sbase, t, c, we, wo);
            else store_chunk<BF16, NPA, VEC>(sbase, t, c, pe, po);
        }
        return;
    }
    double ax[STEPS], vv[STEPS];
#pragma unroll
    for (int q = 0; q < STEPS; ++q) {
        const double a = __shfl_sync(0xffffffffu, a_cur, q);
        ax[q] = int_product(q) ? mul_coef(a, X) : fma(a, x, 0.0);
    }
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        const bool live_k = (k == 0);
#pragma unroll
        for (int q = c * 2 * VEC; q < (c + 1) * 2 * VEC; ++q) {
            vv[q] = live_k ? p1 : 0.0;
            const double tt = fma(ax[q], p1, -p0);
            p0 = p1;
            p1 = tt;
        }
        if (k < 0 && above_hi(p1)) {
            p1 *= 0x1p-512;
            p0 *= 0x1p-512;
            k += 1;
        }
    }
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        if constexpr (BF16) {
            uint32_t we[NPA][4], wo[NPA][4];
#pragma unroll
            for (int v = 0; v < VEC; v += 2) {
                const int q = c * 2 * VEC + 2 * v;
                uint32_t e2[NPA], o2[NPA];
                split_pair_bf16<NPA>(rn_f32(l + q <= L ? vv[q] : 0.0), rn_f32(l + q + 2 <= L ? vv[q + 2] : 0.0), e2);
                split_pair_bf16<NPA>(rn_f32(l + q + 1 <= L ? vv[q + 1] : 0.0), rn_f32(l + q + 3 <= L ? vv[q + 3] : 0.0),
                                     o2);
#pragma unroll
                for (int i = 0; i < NPA; ++i) {
                    we[i][v / 2] = e2[i];
                    wo[i][v / 2] = o2[i];
                }
            }
            store_words<NPA>(sbase, t, c, we, wo);
            continue;
        }
        uint32_t pe[NPA][VEC], po[NPA][VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int q = c * 2 * VEC + 2 * v;
            uint32_t ce[NPA], co[NPA];
            split_pieces<BF16, NPA>(rn_f32(l + q <= L ? vv[q] : 0.0), ce);
            split_pieces<BF16, NPA>(rn_f32(l + q + 1 <= L ? vv[q + 1] : 0.0), co);
#pragma unroll
            for (int i = 0; i < NPA; ++i) {
                pe[i][v] = ce[i];
                po[i][v] = co[i];
            }
        }
        store_chunk<BF16, NPA, VEC>(sbase, t, c, pe, po);
    }
}

constexpr int kWarps = 10;    // 0-3 producers, 4-7 drain, 8 TMA + tensor memory, 9 MMA
constexpr int kPrefetch = 8;  // stages of B tiles prefetched into L2 ahead of their load

// Persistent kernel: CTA c handles work items c, c + gridDim.x, ... where
// item j = (m = j / nrb, ring block rb = j % nrb): heavy (small m) items first.
// MULTI: the items come from the list `items` (request, m, ring block), one
// map per request, each with its own plan (plans[request]) and its own B
// operand, segment table and Delta (mp): many requests of different grids and
// band limits in one launch.
template <bool BF16, int NPA, int NPB, bool MULTI = false>
__global__ void __launch_bounds__(kWarps * 32, 1)
legendre_tc_kernel(const __grid_constant__ DevPlan P, const unsigned char *__restrict__ bbuf,
                   const int *__restrict__ seg_off, float2 *__restrict__ delta, int nmaps, int ncols,
                   int *__restrict__ status, int withhold, const DevPlan *__restrict__ plans,
                   const int4 *__restrict__ items, int nitems_multi, const __grid_constant__ MultiTcPtrs mp)
{
    using C = Cfg<BF16, NPA, NPB>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t base_u32 = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (base_u32 & 1023u)) & 1023u;
    unsigned char *stage0 = smem_raw + pad;
    float2 *stage_d = reinterpret_cast<float2 *>(stage0 + C::NS * C::STAGE_BYTES);  // Delta staging, 4 x 4 KB
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage0 + C::NS * C::STAGE_BYTES + C::STG_BYTES);
    // bars: full_a[NS], full_b[NS], empty[NS], acc_full, acc_empty, mma_drain
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int nrb = (P.npairs + kRows - 1) / kRows;
    const int nitems = MULTI ? nitems_multi : nrb * (P.mmax + 1);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    auto bar_full_a = [&](int s) { return smem_u32(&bars[s]); };
    auto bar_full_b = [&](int s) { return smem_u32(&bars[C::NS + s]); };
    auto bar_empty = [&](int s) { return smem_u32(&bars[2 * C::NS + s]); };
    const uint32_t bar_acc_full = smem_u32(&bars[3 * C::NS]);
    const uint32_t bar_acc_empty = smem_u32(&bars[3 * C::NS + 1]);
    const uint32_t bar_mma_drain = smem_u32(&bars[3 * C::NS + 2]);
    auto a_tile = [&](int s, int par, int piece) {
        return stage0 + s * C::STAGE_BYTES + (par * NPA + piece) * kTileBytes;
    };
    auto b_tile = [&](int s, int par, int piece) {
        return stage0 + s * C::STAGE_BYTES + (C::A_TILES + par * NPB + piece) * kTileBytes;
    };
    // work item -> plan, order m, ring block, B operand, segment table, Delta
    struct Work {
        const DevPlan *Q;
        int m, rb;
        const unsigned char *bb;
        const int *seg;
        float2 *dl;
    };
    auto work_of = [&](int it) {
        Work w;
        if constexpr (MULTI) {
            const int4 v = items[it];
            w.Q = plans + v.x;
            w.m = v.y;
            w.rb = v.z;
            w.bb = static_cast<const unsigned char *>(mp.bbuf[v.x]);
            w.seg = mp.seg[v.x];
            w.dl = static_cast<float2 *>(mp.delta[v.x]);
        } else {
            w.Q = &P;
            w.m = it / nrb;
            w.rb = it - w.m * nrb;
            w.bb = bbuf;
            w.seg = seg_off;
            w.dl = delta;
        }
        return w;
    };
    auto nstages_of = [&](const DevPlan &Q, int m) { return (Q.lmax - m + 1 + C::STEPS - 1) / C::STEPS; };
    // first stage of a work item (evanescent skip: whole 64-degree groups)
    auto first_stage = [&](const DevPlan &Q, int m, int rb) {
        return Q.skip_g ? Q.skip_g[(size_t)m * ((Q.npairs + kRows - 1) / kRows) + rb] * C::GROUP : 0;
    };

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < C::NS; ++s) {
            mbar_init(bar_full_a(s), 4);
            mbar_init(bar_full_b(s), 1);
            mbar_init(bar_empty(s), 1);
        }
        mbar_init(bar_acc_full, 1);
        mbar_init(bar_acc_empty, 4);
        mbar_init(bar_mma_drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        // columns [0, 256): the accumulator of the current 64-degree group, E
        // in [0, ncols) and O in [ncols, 2 ncols); columns [256, 512): the
        // item's FP32 totals in the same arrangement
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    // the CTA's work items: its list of the balanced schedule (the plan's, or
    // the CTA-major item order of a many-request launch), else round robin
    const int *off = MULTI ? mp.cta_off : P.sched_off;
    const bool listed = (MULTI ? mp.ctas : P.sched_ctas) == (int)gridDim.x;
    const int i0 = listed ? off[blockIdx.x] : (int)blockIdx.x;
    const int i1 = listed ? off[blockIdx.x + 1] : nitems;
    const int istep = listed ? 1 : (int)gridDim.x;
    auto item_at = [&](int j) { return (listed && !MULTI) ? P.sched_items[j] : j; };

    if (warp < 4) {
        // ------------------------------------------------------ producers --
        const int t = threadIdx.x;
        uint32_t gs = 0;
        bool ok = true;
        for (int jt = i0; jt < i1 && ok; jt += istep) {
            const int item = item_at(jt);
            const Work w = work_of(item);
            const DevPlan &Q = *w.Q;
            const int m = w.m;
            const int L = Q.lmax;
            const int pair = w.rb * kRows + t;
            const bool live = pair < Q.npairs;
            const int s0 = first_stage(Q, m, w.rb);
            double x = 0.0, p0 = 0.0, p1 = 0.0;
            int k = 0;
            if (live) {
                const size_t o = SHT_IDX(Q.dbg, (size_t)m * Q.npairs + pair, (size_t)(Q.mmax + 1) * Q.npairs, 401);
                x = Q.pair_x[pair];
                if (s0 > 0) {
                    p0 = Q.warm_p0[o];
                    p1 = Q.warm_p1[o];
                    k = Q.warm_k[o];
                } else {
                    p1 = Q.start_v[o];
                    k = Q.start_k[o];
                }
            }
            const XInt X = xint_of(x);
            const long long mofs = (long long)m * (2 * L + 3 - m) / 2;
            const int nst = nstages_of(Q, m);
            int l = m + s0 * C::STEPS;
            // A_{l+1} for the stage's degrees, one per lane, prefetched a stage ahead
            auto coef = [&](int lq) { return (lane < C::STEPS && lq <= L) ? __ldg(&Q.coefA[mofs + (lq - m)]) : 0.0; };
            double a_cur = coef(l + 1 + lane);
            for (int i = s0; i < nst; ++i) {
                const int s = (int)(gs % C::NS);
                const uint32_t ph = (gs / C::NS) & 1u;
                const double a_next = coef(m + (i + 1) * C::STEPS + 1 + lane);
                ok = __all_sync(0xffffffffu, mbar_wait(bar_empty(s), ph ^ 1u, &s_abort));
                if (!ok) break;
                if (__any_sync(0xffffffffu, k < 0))
                    produce_stage<BF16, NPA, true>(a_tile(s, 0, 0), t, x, X, a_cur, l, L, p0, p1, k);
                else
                    produce_stage<BF16, NPA, false>(a_tile(s, 0, 0), t, x, X, a_cur, l, L, p0, p1, k);
                l += C::STEPS;
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_full_a(s));
                ++gs;
                a_cur = a_next;
            }
        }
    } else if (warp < 8) {
        // ----------------------------------------------------------- drain --
        const int quad = warp - 4;
        const int row = quad * 32 + lane;  // tensor-memory lane = ring pair in the block
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        uint32_t gg = 0;
        bool ok = true;
        for (int jt = i0; jt < i1 && ok; jt += istep) {
            const int item = item_at(jt);
            const Work w = work_of(item);
            const DevPlan &Q = *w.Q;
            const int m = w.m;
            const int pair = w.rb * kRows + row;
            const int ngroups = (nstages_of(Q, m) + C::GROUP - 1) / C::GROUP - first_stage(Q, m, w.rb) / C::GROUP;
            for (int g = 0; g < ngroups; ++g) {
                ok = __all_sync(0xffffffffu, mbar_wait(bar_acc_full, gg & 1u, &s_abort));
                if (!ok) break;
                tc_fence_after();
                // totals (columns 256 + c) = accumulator (g = 0), else totals + accumulator,
                // added in FP32 with rounding to nearest, 32 columns at a time
                for (int c0 = 0; c0 < 2 * ncols; c0 += 32) {
                    uint32_t v[32], t[32];
                    SHT_CHECK(Q.dbg, c0 + 32 <= 256, 402);
                    tmem_ld32_async(tmem + lane_base + (uint32_t)c0, v);
                    if (g > 0) tmem_ld32_async(tmem + lane_base + (uint32_t)(256 + c0), t);
                    tmem_wait_ld();
                    if (g > 0) {
                        // two FP32 adds (round to nearest) per instruction
#pragma unroll
                        for (int j = 0; j < 32; j += 2) {
                            const unsigned long long a = ((unsigned long long)t[j + 1] << 32) | t[j];
                            const unsigned long long b = ((unsigned long long)v[j + 1] << 32) | v[j];
                            unsigned long long d;
                            asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
                            v[j] = (uint32_t)d;
                            v[j + 1] = (uint32_t)(d >> 32);
                        }
                    }
                    tmem_st32(tmem + lane_base + (uint32_t)(256 + c0), v);
                    tmem_wait_st();
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_acc_empty);
                ++gg;
            }
            if (!ok) break;
            // Delta_m(north) = E + O, Delta_m(south) = E - O for the warp's 32
            // rows; Delta is [ring][m][map].  Per block of 16 maps (columns
            // 32 k .. 32 k + 31 of E and of O) the warp reads its rows'
            // totals, and each row's 128 bytes of N (then S) go through the
            // warp's staging buffer (row = lane, element c at c ^ (lane & 15):
            // no bank conflicts) and out as 16-byte stores, four rows per
            // instruction.
            {
                int2 rr = make_int2(-1, -1);
                if (pair < Q.npairs) rr = Q.pair_ring[pair];
                const int M1 = Q.mmax + 1;
                const bool vec = (nmaps & 1) == 0;
                float2 *stg = stage_d + quad * (32 * 16);
                for (int k = 0; 32 * k < ncols; ++k) {
                    uint32_t e[32], o[32];
                    tmem_ld32_async(tmem + lane_base + (uint32_t)(256 + 32 * k), e);
                    tmem_ld32_async(tmem + lane_base + (uint32_t)(256 + ncols + 32 * k), o);
                    tmem_wait_ld();
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            const float er = __uint_as_float(e[2 * c]), ei = __uint_as_float(e[2 * c + 1]);
                            const float orr = __uint_as_float(o[2 * c]), oi = __uint_as_float(o[2 * c + 1]);
                            stg[lane * 16 + (c ^ (lane & 15))] =
                                side == 0 ? make_float2(er + orr, (m == 0) ? 0.f : ei + oi)
                                          : make_float2(er - orr, (m == 0) ? 0.f : ei - oi);
                        }
                        __syncwarp();
                        const int sg = lane & 7;  // maps 16 k + 2 sg and + 1
                        const int b = 16 * k + 2 * sg;
#pragma unroll
                        for (int it = 0; it < 8; ++it) {
                            const int rw = it * 4 + (lane >> 3);
                            const int ring = __shfl_sync(0xffffffffu, side == 0 ? rr.x : rr.y, rw);
                            const float2 v0 = stg[rw * 16 + ((2 * sg) ^ (rw & 15))];
                            const float2 v1 = stg[rw * 16 + ((2 * sg + 1) ^ (rw & 15))];
                            if (ring >= 0) {
                                // maps b, b + 1 are stored only where they exist (b < nmaps)
                                SHT_CHECK(Q.dbg, ring < Q.nrings && m < M1, 403);
                                float2 *d = w.dl + ((size_t)ring * M1 + m) * nmaps + b;
                                if (vec && b + 1 < nmaps) {
                                    *reinterpret_cast<float4 *>(d) = make_float4(v0.x, v0.y, v1.x, v1.y);
                                } else {
                                    if (b < nmaps) d[0] = v0;
                                    if (b + 1 < nmaps) d[1] = v1;
                                }
                            }
                        }
                        __syncwarp();
                    }
                }
            }
        }
    } else if (warp == 8) {
        // ------------------------------------------------------ B loads --
        // The operand prep wrote the B tiles of every (m, stage) as one
        // contiguous block in the shared-memory image ([parity][piece] tiles
        // of 4 KB, swizzled), so one bulk copy fills a stage.
        if (lane == 0) {
            constexpr uint32_t SB = (uint32_t)C::B_TILES * kTileBytes;
            uint32_t gs = 0;
            bool ok = true;
            for (int jt = i0; jt < i1 && ok; jt += istep) {
                const int item = item_at(jt);
                const Work w = work_of(item);
            const DevPlan &Q = *w.Q;
            const int m = w.m;
            const int L = Q.lmax;
                const unsigned char *blk = w.bb + (size_t)(w.seg[2 * m] / C::STEPS) * SB;
                const int nst = nstages_of(Q, m);
                const int s0 = first_stage(Q, m, w.rb);
                // the item's stages stay inside its (m, parity) segments
                SHT_CHECK(Q.dbg, w.seg[2 * m] % C::STEPS == 0 && nst * (C::STEPS / 2) <= w.seg[2 * m + 1] - w.seg[2 * m] + 0,
                          404);
                SHT_CHECK(Q.dbg, s0 >= 0 && s0 <= nst, 405);
                for (int i = s0; i < s0 + kPrefetch && i < nst; ++i) bulk_prefetch_l2(blk + (size_t)i * SB, SB);
                for (int i = s0; i < nst; ++i) {
                    const int s = (int)(gs % C::NS);
                    const uint32_t ph = (gs / C::NS) & 1u;
                    if (i + kPrefetch < nst) bulk_prefetch_l2(blk + (size_t)(i + kPrefetch) * SB, SB);
                    if ((int)gs == withhold && blockIdx.x == 0) {
                        ++gs;  // test hook: this stage's copy is never issued
                        continue;
                    }
                    if (!mbar_wait(bar_empty(s), ph ^ 1u, &s_abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(bar_full_b(s), SB);
                    bulk_load(smem_u32(b_tile(s, 0, 0)), blk + (size_t)i * SB, SB, bar_full_b(s));
                    ++gs;
                }
            }
            if (s_abort) {
                // let the copies in flight land before the CTA exits
                const uint32_t first = gs > (uint32_t)C::NS ? gs - C::NS : 0u;
                for (uint32_t j = first; j < gs; ++j) mbar_drain(bar_full_b((int)(j % C::NS)), (j / C::NS) & 1u);
            }
        }
    } else {
        // ----------------------------------------------------------- MMA --
        if (lane == 0) {
            const uint32_t id = idesc<BF16>(ncols);
            uint32_t gs = 0, gg = 0;
            bool ok = true, issued = false;
            for (int jt = i0; jt < i1 && ok; jt += istep) {
                const int item = item_at(jt);
                const Work w = work_of(item);
            const DevPlan &Q = *w.Q;
            const int m = w.m;
            const int L = Q.lmax;
                const int nst = nstages_of(Q, m);
                for (int i0 = first_stage(Q, m, w.rb); i0 < nst && ok; i0 += C::GROUP) {
                    // the drain has read the previous group's accumulator
                    if (!mbar_wait(bar_acc_empty, (gg & 1u) ^ 1u, &s_abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int i1 = min(nst, i0 + C::GROUP);
                    for (int i = i0; i < i1; ++i) {
                        const int s = (int)(gs % C::NS);
                        const uint32_t ph = (gs / C::NS) & 1u;
                        if (!mbar_wait(bar_full_a(s), ph, &s_abort) || !mbar_wait(bar_full_b(s), ph, &s_abort)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        SHT_CHECK(Q.dbg, 2 * ncols <= 256 && s < C::NS, 406);
#pragma unroll
                        for (int par = 0; par < 2; ++par) {
                            const uint32_t d = tmem + (uint32_t)(par * ncols);
#pragma unroll
                            for (int pr = 0; pr < C::NPROD; ++pr) {
                                int ia, ib;
                                product_pieces<NPA, NPB>(pr, ia, ib);
                                const uint64_t ad = sdesc_sw32(smem_u32(a_tile(s, par, ia)));
                                const uint64_t bd = sdesc_sw32(smem_u32(b_tile(s, par, ib)));
                                tc_mma<BF16>(d, ad, bd, id, (i > i0 || pr > 0) ? 1u : 0u);
                            }
                        }
                        issued = true;
                        tc_commit(bar_empty(s));
                        ++gs;
                    }
                    if (!ok) break;
                    tc_commit(bar_acc_full);
                    ++gg;
                }
            }
            if (!ok && issued) {
                // wait (bounded) for the MMAs already issued before tensor memory is freed
                tc_commit(bar_mma_drain);
                mbar_drain(bar_mma_drain, 0u);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
    }
    if (threadIdx.x == 0 && s_abort) atomicExch(status, SHT_ETIMEOUT);
}

// ------------------------------------------------ streaming (cached) kernel --
// The same contraction with the A tiles read from the plan-time Lambda
// operand (lambda_build_kernel) instead of computed: no producer warps, so
// the drain keeps its FP32 totals in registers and shared memory holds only
// the stage ring, NS_STREAM stages deep.  Persistent, one CTA per SM:
//   warps 0-7  drain: warp w reads tensor-memory lanes 32 (w % 4) .. + 32 and
//              the 32-column chunks q = 2 j + w / 4 of E and O; after every 64
//              degrees it adds the finished accumulator set into its register
//              totals (FP32, round to nearest: the order and rounding of the
//              recurrence kernel's drain, so the results are bit-identical),
//              and at the end of an item writes Delta for its maps;
//   warp 8     tensor memory, and one bulk copy each for the stage's A and B
//              tiles (no L2 prefetch: with NS stages of bulk copies in
//              flight it only competed with them);
//   warp 9     the MMAs, as in legendre_tc_kernel.
template <bool BF16, int NPA, int NPB>
struct StreamCfg {
    using C = Cfg<BF16, NPA, NPB>;
    static constexpr int STG_BYTES = 8 * 32 * 16 * 8;  // per drain warp: 32 rows x 16 float2
    static constexpr int NS = (227 * 1024 - 1024 - 256 - STG_BYTES) / C::STAGE_BYTES;  // 4 (48 KB) or 6 (32 KB)
    static constexpr int SMEM = NS * C::STAGE_BYTES + STG_BYTES + 1024 /* align */ + 256 /* barriers */;
};

template <bool BF16, int NPA, int NPB>
__global__ void __launch_bounds__(kWarps * 32, 1)
legendre_tc_stream_kernel(const DevPlan P, const unsigned char *__restrict__ bbuf,
                          const unsigned char *__restrict__ acache, const int *__restrict__ seg_off,
                          float2 *__restrict__ delta, int nmaps, int ncols, int *__restrict__ status, int withhold)
{
    using C = Cfg<BF16, NPA, NPB>;
    constexpr int NS = StreamCfg<BF16, NPA, NPB>::NS;
    constexpr uint32_t SA = (uint32_t)C::A_TILES * kTileBytes;
    constexpr uint32_t SB = (uint32_t)C::B_TILES * kTileBytes;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t base_u32 = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (base_u32 & 1023u)) & 1023u;
    unsigned char *stage0 = smem_raw + pad;
    float2 *stage_d = reinterpret_cast<float2 *>(stage0 + NS * C::STAGE_BYTES);  // Delta staging, 8 x 4 KB
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage0 + NS * C::STAGE_BYTES + StreamCfg<BF16, NPA, NPB>::STG_BYTES);
    // bars: full[NS], empty[NS], set_full[2], set_empty[2], mma_drain
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int L = P.lmax;
    const int nrb = (P.npairs + kRows - 1) / kRows;
    const int nitems = nrb * (P.mmax + 1);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    auto bar_full = [&](int s) { return smem_u32(&bars[s]); };
    auto bar_empty = [&](int s) { return smem_u32(&bars[NS + s]); };
    auto bar_set_full = [&](int j) { return smem_u32(&bars[2 * NS + j]); };
    auto bar_set_empty = [&](int j) { return smem_u32(&bars[2 * NS + 2 + j]); };
    const uint32_t bar_mma_drain = smem_u32(&bars[2 * NS + 4]);
    auto a_tile = [&](int s, int par, int piece) {
        return stage0 + s * C::STAGE_BYTES + (par * NPA + piece) * kTileBytes;
    };
    auto b_tile = [&](int s, int par, int piece) {
        return stage0 + s * C::STAGE_BYTES + (C::A_TILES + par * NPB + piece) * kTileBytes;
    };
    auto nstages_of = [&](int m) { return (L - m + 1 + C::STEPS - 1) / C::STEPS; };
    // first stage of a work item (evanescent skip: whole 64-degree groups)
    auto first_stage = [&](int item) { return P.skip_g ? P.skip_g[item] * C::GROUP : 0; };

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < NS; ++s) {
            mbar_init(bar_full(s), 1);
            mbar_init(bar_empty(s), 1);
        }
        for (int j = 0; j < 2; ++j) {
            mbar_init(bar_set_full(j), 1);
            mbar_init(bar_set_empty(j), 8);
        }
        mbar_init(bar_mma_drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const bool listed = P.sched_ctas == (int)gridDim.x;
    const int i0 = listed ? P.sched_off[blockIdx.x] : (int)blockIdx.x;
    const int i1 = listed ? P.sched_off[blockIdx.x + 1] : nitems;
    const int istep = listed ? 1 : (int)gridDim.x;
    auto item_at = [&](int j) { return listed ? P.sched_items[j] : j; };

    if (warp < 8) {
        // ----------------------------------------------------------- drain --
        const int quad = warp & 3;
        const int half = warp >> 2;
        const int row = quad * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        float te[2][32], to[2][32];  // totals of chunks q = 2 j + half of E and O
        uint32_t gg = 0;
        bool ok = true;
        for (int jt = i0; jt < i1 && ok; jt += istep) {
            const int item = item_at(jt);
            const int m = item / nrb;
            const int pair = (item % nrb) * kRows + row;
            const int ngroups = (nstages_of(m) + C::GROUP - 1) / C::GROUP - first_stage(item) / C::GROUP;
            for (int g = 0; g < ngroups; ++g) {
                const int set = (int)(gg & 1u);
                ok = __all_sync(0xffffffffu, mbar_wait(bar_set_full(set), (gg >> 1) & 1u, &s_abort));
                if (!ok) break;
                tc_fence_after();
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int q = 2 * j + half;
                    if (32 * q < ncols) {
                        uint32_t v[32];
                        tmem_ld32(tmem + lane_base + (uint32_t)(256 * set + 32 * q), v);
#pragma unroll
                        for (int c = 0; c < 32; ++c) te[j][c] = (g == 0) ? __uint_as_float(v[c]) : te[j][c] + __uint_as_float(v[c]);
                        tmem_ld32(tmem + lane_base + (uint32_t)(256 * set + ncols + 32 * q), v);
#pragma unroll
                        for (int c = 0; c < 32; ++c) to[j][c] = (g == 0) ? __uint_as_float(v[c]) : to[j][c] + __uint_as_float(v[c]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_set_empty(set));
                ++gg;
            }
            if (!ok) break;
            // Delta_m(north) = E + O, Delta_m(south) = E - O for the warp's 32
            // rows and its maps; Delta is [ring][m][map].  Each block of 16
            // maps of a row (128 contiguous bytes) goes through the warp's
            // staging buffer (row = lane, element c at c ^ (lane & 15): no bank
            // conflicts) and out as 16-byte stores, four rows per instruction.
            int2 rr = make_int2(-1, -1);
            if (pair < P.npairs) rr = P.pair_ring[pair];
            const int M1 = P.mmax + 1;
            const bool vec = (nmaps & 1) == 0;
            float2 *stg = stage_d + warp * (32 * 16);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int q = 2 * j + half;  // columns 32 q .. 32 q + 31 = maps 16 q .. 16 q + 15
                if (32 * q >= ncols) continue;
#pragma unroll
                for (int side = 0; side < 2; ++side) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const float er = te[j][2 * c], ei = te[j][2 * c + 1];
                        const float orr = to[j][2 * c], oi = to[j][2 * c + 1];
                        stg[lane * 16 + (c ^ (lane & 15))] =
                            side == 0 ? make_float2(er + orr, (m == 0) ? 0.f : ei + oi)
                                      : make_float2(er - orr, (m == 0) ? 0.f : ei - oi);
                    }
                    __syncwarp();
                    const int sg = lane & 7;
                    const int b = 16 * q + 2 * sg;
#pragma unroll
                    for (int it = 0; it < 8; ++it) {
                        const int rw = it * 4 + (lane >> 3);
                        const int ring = __shfl_sync(0xffffffffu, side == 0 ? rr.x : rr.y, rw);
                        const float2 v0 = stg[rw * 16 + ((2 * sg) ^ (rw & 15))];
                        const float2 v1 = stg[rw * 16 + ((2 * sg + 1) ^ (rw & 15))];
                        if (ring >= 0) {
                            float2 *d = delta + ((size_t)ring * M1 + m) * nmaps + b;
                            if (vec && b + 1 < nmaps) {
                                *reinterpret_cast<float4 *>(d) = make_float4(v0.x, v0.y, v1.x, v1.y);
                            } else {
                                if (b < nmaps) d[0] = v0;
                                if (b + 1 < nmaps) d[1] = v1;
                            }
                        }
                    }
                    __syncwarp();
                }
            }
        }
    } else if (warp == 8) {
        // ---------------------------------------------------- A + B loads --
        if (lane == 0) {
            uint32_t gs = 0;
            bool ok = true;
            for (int jt = i0; jt < i1 && ok; jt += istep) {
                const int item = item_at(jt);
                const int m = item / nrb;
                const size_t st0 = (size_t)(seg_off[2 * m] / C::STEPS);  // stages of the orders below m
                const int nst = nstages_of(m);
                const unsigned char *bblk = bbuf + st0 * SB;
                const unsigned char *ablk = acache + (st0 * nrb + (size_t)(item % nrb) * nst) * SA;
                for (int i = first_stage(item); i < nst; ++i) {
                    const int s = (int)(gs % NS);
                    const uint32_t ph = (gs / NS) & 1u;
                    if ((int)gs == withhold && blockIdx.x == 0) {
                        ++gs;  // test hook: this stage's copies are never issued
                        continue;
                    }
                    if (!mbar_wait(bar_empty(s), ph ^ 1u, &s_abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(bar_full(s), SA + SB);
                    bulk_load(smem_u32(a_tile(s, 0, 0)), ablk + (size_t)i * SA, SA, bar_full(s));
                    bulk_load(smem_u32(b_tile(s, 0, 0)), bblk + (size_t)i * SB, SB, bar_full(s));
                    ++gs;
                }
            }
            if (s_abort) {
                const uint32_t first = gs > (uint32_t)NS ? gs - NS : 0u;
                for (uint32_t j = first; j < gs; ++j) mbar_drain(bar_full((int)(j % NS)), (j / NS) & 1u);
            }
        }
    } else {
        // ----------------------------------------------------------- MMA --
        if (lane == 0) {
            const uint32_t id = idesc<BF16>(ncols);
            uint32_t gs = 0, gg = 0;
            bool ok = true, issued = false;
            for (int jt = i0; jt < i1 && ok; jt += istep) {
                const int item = item_at(jt);
                const int m = item / nrb;
                const int nst = nstages_of(m);
                for (int i0 = first_stage(item); i0 < nst && ok; i0 += C::GROUP) {
                    const int set = (int)(gg & 1u);
                    if (!mbar_wait(bar_set_empty(set), ((gg >> 1) & 1u) ^ 1u, &s_abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int i1 = min(nst, i0 + C::GROUP);
                    for (int i = i0; i < i1; ++i) {
                        const int s = (int)(gs % NS);
                        const uint32_t ph = (gs / NS) & 1u;
                        if (!mbar_wait(bar_full(s), ph, &s_abort)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        SHT_CHECK(P.dbg, 256 * set + 2 * ncols <= 512 && s < NS, 407);
#pragma unroll
                        for (int par = 0; par < 2; ++par) {
                            const uint32_t d = tmem + (uint32_t)(256 * set + par * ncols);
#pragma unroll
                            for (int pr = 0; pr < C::NPROD; ++pr) {
                                int ia, ib;
                                product_pieces<NPA, NPB>(pr, ia, ib);
                                const uint64_t ad = sdesc_sw32(smem_u32(a_tile(s, par, ia)));
                                const uint64_t bd = sdesc_sw32(smem_u32(b_tile(s, par, ib)));
                                tc_mma<BF16>(d, ad, bd, id, (i > i0 || pr > 0) ? 1u : 0u);
                            }
                        }
                        issued = true;
                        tc_commit(bar_empty(s));
                        ++gs;
                    }
                    if (!ok) break;
                    tc_commit(bar_set_full(set));
                    ++gg;
                }
            }
            if (!ok && issued) {
                tc_commit(bar_mma_drain);
                mbar_drain(bar_mma_drain, 0u);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
    }
    if (threadIdx.x == 0 && s_abort) atomicExch(status, SHT_ETIMEOUT);
}

// ------------------------------------------------------------ operand prep --
// B[c][seg(m, par) + k] = pieces of C_l a_lm(map c/2, re or im), l = m + par + 2k,
// zero for l > lmax, for maps beyond nmaps and for Im of m = 0.
// B operand image: for every (m, stage) a contiguous block of 2 x NPB tiles
// ([parity][piece], 4 KB each) laid out exactly as the kernel's shared-memory
// B tiles: row c (= 2 map + {re, im}) of 32 bytes holds the stage's KC
// degrees of one parity, 16-byte chunks swizzled by bit 2 of the row.  Entry
// (par, c, k) holds the pieces of C_l a_lm(map c/2, re or im), l = m + par + 2k,
// zero for l > lmax, for maps beyond nmaps and for Im of m = 0.
// The pieces of order m's segment; the (stage, par, c, kk) elements are split
// over threads t0, t0 + tstep, ... (each element is computed on its own, so
// the split does not change a bit).
template <bool BF16, int NPB>
__device__ __forceinline__ void prep_b_order(const DevPlan &P, const double2 *__restrict__ alm,
                                             const int *__restrict__ seg_off, unsigned char *__restrict__ bout,
                                             int nmaps, int ncols, int m, int t0, int tstep)
{
    constexpr int KC = BF16 ? 16 : 8;
    constexpr int ESZ = BF16 ? 2 : 4;
    constexpr size_t SB = (size_t)2 * NPB * kTileBytes;
    const int L = P.lmax;
    const int nst = (L - m + 1 + 2 * KC - 1) / (2 * KC);
    const long long mofs = (long long)m * (2 * L + 3 - m) / 2;
    unsigned char *blk = bout + (size_t)(seg_off[2 * m] / (2 * KC)) * SB;
    const int total = nst * 2 * ncols * KC;  // (stage, par, c, kk), kk fastest
    for (int idx = t0; idx < total; idx += tstep) {
        const int kk = idx % KC;
        const int c = (idx / KC) % ncols;
        const int par = (idx / (KC * ncols)) % 2;
        const int i = idx / (KC * ncols * 2);
        const int l = m + par + 2 * (i * KC + kk);
        const int b = c >> 1;
        float v = 0.f;
        if (l <= L && b < nmaps && !(m == 0 && (c & 1))) {
            const double2 a = alm[(size_t)b * P.nalm + mofs + (l - m)];
            v = rn_f32(P.coefC[mofs + (l - m)] * ((c & 1) ? a.y : a.x));
        }
        uint32_t pc[NPB];
        split_pieces<BF16, NPB>(v, pc);
        const int byte = kk * ESZ;
        const int off = c * kRowBytes + ((((byte >> 4) ^ ((c >> 2) & 1))) << 4) + (byte & 15);
#pragma unroll
        for (int q = 0; q < NPB; ++q) {
            unsigned char *dst = blk + (size_t)i * SB + (size_t)(par * NPB + q) * kTileBytes + off;
            if (BF16)
                *reinterpret_cast<uint16_t *>(dst) = (uint16_t)(pc[q] >> 16);
            else
                *reinterpret_cast<uint32_t *>(dst) = pc[q];
        }
    }
}

// Operand prep of many one-map requests in one launch: block i converts order
// items[i].y of request items[i].x into that request's B operand image.
template <bool BF16, int NPB>
__global__ void prep_b_multi_kernel(const DevPlan *__restrict__ plans, const int2 *__restrict__ items,
                                    const __grid_constant__ MultiTcPtrs mp)
{
    const int2 it = items[blockIdx.x];
    prep_b_order<BF16, NPB>(plans[it.x], static_cast<const double2 *>(mp.alm[it.x]), mp.seg[it.x],
                            static_cast<unsigned char *>(const_cast<void *>(mp.bbuf[it.x])), 1, tc_ncols(1), it.y,
                            threadIdx.x, blockDim.x);
}

// The same operand image, one CTA per (stage i, order m): the stage's 2 KC
// degrees of every map are read once with coalesced loads (512 contiguous
// bytes per map for BF16), multiplied by C_l and rounded to FP32 into shared
// memory (row c = 2 map + {re, im}, padded to avoid bank conflicts), then each
// thread turns one half row (parity, c, 16-byte half) into the half rows of
// every piece, written as 16-byte stores.  Same values as prep_b_order.
template <bool BF16, int NPB>
__global__ void __launch_bounds__(256)
prep_b_stage_kernel(const DevPlan P, const double2 *__restrict__ alm, const int *__restrict__ seg_off,
                    unsigned char *__restrict__ bout, int nmaps, int ncols)
{
    constexpr int KC = BF16 ? 16 : 8;
    constexpr int STEPS = 2 * KC;
    constexpr int VEC = BF16 ? 8 : 4;  // values per 16-byte half row
    constexpr size_t SB = (size_t)2 * NPB * kTileBytes;
    __shared__ float sv[128][STEPS + 1];
    const int L = P.lmax;
    const int m = blockIdx.y, i = blockIdx.x;
    const int nst = (L - m + 1 + STEPS - 1) / STEPS;
    if (i >= nst) return;
    const long long mofs = (long long)m * (2 * L + 3 - m) / 2;
    const int l0 = m + STEPS * i;
    SHT_CHECK(P.dbg, ncols <= 128, 408);
    for (int e = threadIdx.x; e < (ncols >> 1) * STEPS; e += blockDim.x) {
        const int b = e / STEPS, o = e - b * STEPS, l = l0 + o;
        float re = 0.f, im = 0.f;
        if (l <= L && b < nmaps) {
            const double c = __ldg(&P.coefC[mofs + (l - m)]);
            const double2 a = __ldg(&alm[(size_t)b * P.nalm + mofs + (l - m)]);
            re = rn_f32(c * a.x);
            if (m != 0) im = rn_f32(c * a.y);
        }
        sv[2 * b][o] = re;
        sv[2 * b + 1][o] = im;
    }
    __syncthreads();
    unsigned char *blk = bout + (size_t)(seg_off[2 * m] / STEPS + i) * SB;
    for (int w = threadIdx.x; w < 4 * ncols; w += blockDim.x) {
        const int h = w & 1, c = (w >> 1) % ncols, par = (w >> 1) / ncols;
        uint32_t words[NPB][4];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            uint32_t pc[NPB];
            split_pieces<BF16, NPB>(sv[c][par + 2 * (VEC * h + v)], pc);
#pragma unroll
            for (int q = 0; q < NPB; ++q) {
                if (BF16) {
                    if (v & 1)
                        words[q][v >> 1] |= pc[q] & 0xFFFF0000u;
                    else
                        words[q][v >> 1] = pc[q] >> 16;
                } else {
                    words[q][v] = pc[q];
                }
            }
        }
        const int off = c * kRowBytes + ((h ^ ((c >> 2) & 1)) << 4);
#pragma unroll
        for (int q = 0; q < NPB; ++q)
            *reinterpret_cast<uint4 *>(blk + (size_t)(par * NPB + q) * kTileBytes + off) =
                make_uint4(words[q][0], words[q][1], words[q][2], words[q][3]);
    }
}

template <bool BF16, int NPA, int NPB>
cudaError_t run_prep(const DevPlan &P, const TcWork &W, const double2 *alm, int nmaps, cudaStream_t st)
{
    constexpr int STEPS = BF16 ? 32 : 16;
    const int ncols = tc_ncols(nmaps);
    const int *seg = BF16 ? W.seg_bf16 : W.seg_tf32;
    dim3 grid((P.lmax + 1 + STEPS - 1) / STEPS, P.mmax + 1);  // stages of order 0, the most
    prep_b_stage_kernel<BF16, NPB>
        <<<grid, 256, 0, st>>>(P, alm, seg, static_cast<unsigned char *>(W.bbuf), nmaps, ncols);
    return cudaGetLastError();
}

// ------------------------------------------------------ evanescent skip --
// Per (m, ring block): the first 64-degree group containing a degree whose
// recurrence value is representable in FP32 (exponent k = 0 and
// |p_l| >= 2^-126) in any ring of the block, and each ring's recurrence state
// at the start of that group.  The recurrence is the producers' (same fused
// operations), rescaled as soon as |p| > 2^256 while k < 0; rescaling by 2^-512
// is exact, so a producer that starts from this state computes the same values
// as one that starts at degree m, and the values it skips would all have
// rounded to zero.  At least one group is kept per item.  pair_lim[pair]
// becomes 1 + the largest m at which the pair has a representable value (its
// Delta is exactly zero at every larger order).  One CTA of 128 threads per
// (ring block, m).
__global__ void __launch_bounds__(kRows)
warm_start_kernel(const DevPlan P, int *__restrict__ skip_g, double *__restrict__ wp0, double *__restrict__ wp1,
                  int *__restrict__ wk, int *__restrict__ pair_lim)
{
    __shared__ int s_first;
    const int L = P.lmax;
    const int nrb = (P.npairs + kRows - 1) / kRows;
    const int rb = blockIdx.x;
    const int m = blockIdx.y;
    const int t = threadIdx.x;
    const int pair = rb * kRows + t;
    const bool live = pair < P.npairs;
    const long long mofs = (long long)m * (2 * L + 3 - m) / 2;
    const double x = live ? P.pair_x[pair] : 0.0;
    const double v0 = live ? P.start_v[(size_t)m * P.npairs + pair] : 0.0;
    const int k0 = live ? P.start_k[(size_t)m * P.npairs + pair] : 0;
    if (t == 0) s_first = L + 1;
    __syncthreads();
    // pass 1: first representable degree of this ring
    {
        double p0 = 0.0, p1 = v0;
        int k = k0;
        for (int l = m; l <= L && live; ++l) {
            if (k == 0 && fabs(p1) >= 0x1p-126) {
                atomicMin(&s_first, l);
                atomicMax(&pair_lim[pair], m + 1);
                break;
            }
            const double a = (l + 1 <= L) ? __ldg(&P.coefA[mofs + (l + 1 - m)]) : 0.0;
            const double tt = fma(fma(a, x, 0.0), p1, -p0);
            p0 = p1;
            p1 = tt;
            if (k < 0 && above_hi(p1)) {
                p1 *= 0x1p-512;
                p0 *= 0x1p-512;
                k += 1;
            }
        }
    }
    __syncthreads();
    const int ngroups = (L - m + 1 + 63) / 64;
    const int g0 = min((s_first - m) / 64, ngroups - 1);
    if (t == 0) skip_g[(size_t)m * nrb + rb] = g0;
    // pass 2: the state at degree m + 64 g0
    if (!live) return;
    double p0 = 0.0, p1 = v0;
    int k = k0;
    for (int l = m; l < m + 64 * g0; ++l) {
        const double a = __ldg(&P.coefA[mofs + (l + 1 - m)]);
        const double tt = fma(fma(a, x, 0.0), p1, -p0);
        p0 = p1;
        p1 = tt;
        if (k < 0 && above_hi(p1)) {
            p1 *= 0x1p-512;
            p0 *= 0x1p-512;
            k += 1;
        }
    }
    const size_t o = (size_t)m * P.npairs + pair;
    wp0[o] = p0;
    wp1[o] = p1;
    wk[o] = k;
}

// ------------------------------------------------- plan-time Lambda operand --
// The A tiles of every (m, ring block rb, stage i) exactly as the producers
// write them into shared memory (same recurrence, same rounding, same pieces,
// same swizzle), one contiguous block of 2 x NPA tiles per stage at
//   ((stages of the orders below m) x nrb + rb x nstages(m) + i) x block size,
// so that a cached launch copies a stage with one bulk copy and gives results
// identical to the recurrence launch.  One CTA of 128 threads per (rb, m).
template <bool BF16, int NPA>
__global__ void __launch_bounds__(kRows)
lambda_build_kernel(const DevPlan P, const int *__restrict__ seg_off, unsigned char *__restrict__ aout)
{
    constexpr int STEPS = BF16 ? 32 : 16;
    constexpr size_t SA = (size_t)2 * NPA * kTileBytes;
    const int L = P.lmax;
    const int nrb = (P.npairs + kRows - 1) / kRows;
    const int rb = blockIdx.x;
    const int m = blockIdx.y;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int pair = rb * kRows + t;
    // stages before the item's first (evanescent skip) are never read: not written
    const int s0 = P.skip_g ? P.skip_g[m * nrb + rb] * (64 / STEPS) : 0;
    double x = 0.0, p0 = 0.0, p1 = 0.0;
    int k = 0;
    if (pair < P.npairs) {
        const size_t o = (size_t)m * P.npairs + pair;
        x = P.pair_x[pair];
        if (s0 > 0) {
            p0 = P.warm_p0[o];
            p1 = P.warm_p1[o];
            k = P.warm_k[o];
        } else {
            p1 = P.start_v[o];
            k = P.start_k[o];
        }
    }
    const XInt X = xint_of(x);
    const long long mofs = (long long)m * (2 * L + 3 - m) / 2;
    const int nst = (L - m + 1 + STEPS - 1) / STEPS;
    unsigned char *blk = aout + ((size_t)(seg_off[2 * m] / STEPS) * nrb + (size_t)rb * nst) * SA;
    auto coef = [&](int lq) { return (lane < STEPS && lq <= L) ? __ldg(&P.coefA[mofs + (lq - m)]) : 0.0; };
    int l = m + s0 * STEPS;
    for (int i = s0; i < nst; ++i) {
        const double a_cur = coef(l + 1 + lane);
        if (__any_sync(0xffffffffu, k < 0))
            produce_stage<BF16, NPA, true>(blk + (size_t)i * SA, t, x, X, a_cur, l, L, p0, p1, k);
        else
            produce_stage<BF16, NPA, false>(blk + (size_t)i * SA, t, x, X, a_cur, l, L, p0, p1, k);
        l += STEPS;
    }
}

template <bool STREAM, typename K>
cudaError_t launch_persistent(K kern, int smem, const DevPlan &P, const TcWork &W, const void *acache,
                             const int *seg, float2 *delta, int nmaps, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const long long nitems = (long long)((P.npairs + kRows - 1) / kRows) * (P.mmax + 1);
    const int grid = (int)std::min<long long>(nitems, nsm);  // persistent: one CTA per SM
    const unsigned char *b = static_cast<const unsigned char *>(W.bbuf);
    const int ncols = tc_ncols(nmaps);
    if constexpr (STREAM) {
        kern<<<grid, kWarps * 32, smem, st>>>(P, b, static_cast<const unsigned char *>(acache), seg, delta, nmaps,
                                              ncols, W.status, W.withhold);
    } else {
        static const MultiTcPtrs none{};
        kern<<<grid, kWarps * 32, smem, st>>>(P, b, seg, delta, nmaps, ncols, W.status, W.withhold, nullptr, nullptr,
                                              0, none);
    }
    return cudaGetLastError();
}

template <bool BF16, int NPA, int NPB>
cudaError_t run_main_multi(const DevPlan &P, const DevPlan *plans_dev, const int4 *items, int nitems,
                           const MultiTcPtrs &mp, int *status, cudaStream_t st)
{
    using C = Cfg<BF16, NPA, NPB>;
    auto kern = legendre_tc_kernel<BF16, NPA, NPB, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = std::min(nitems, nsm);  // persistent: one CTA per SM
    kern<<<grid, kWarps * 32, C::SMEM, st>>>(P, nullptr, nullptr, nullptr, 1, tc_ncols(1), status, -1, plans_dev,
                                             items, nitems, mp);
    return cudaGetLastError();
}

template <bool BF16, int NPA, int NPB>
cudaError_t run_main(const DevPlan &P, const TcWork &W, const void *acache, float2 *delta, int nmaps,
                     cudaStream_t st)
{
    const int *seg = BF16 ? W.seg_bf16 : W.seg_tf32;
    if (acache)
        return launch_persistent<true>(legendre_tc_stream_kernel<BF16, NPA, NPB>, StreamCfg<BF16, NPA, NPB>::SMEM, P, W,
                                 acache, seg, delta, nmaps, st);
    return launch_persistent<false>(legendre_tc_kernel<BF16, NPA, NPB>, Cfg<BF16, NPA, NPB>::SMEM, P, W, nullptr, seg, delta,
                             nmaps, st);
}

// ------------------------------------------------ tensor-core transpose --
// Legendre step of the transpose (map2alm_adjoint, Eq. DeltaDef transposed),
// BF16 forms, from the plan-time Lambda operand:
//     g_lm = c_m C_l sum_pairs p_l(x) (q_N + (-1)^{l-m} q_S)(m),  c_0 = 1, c_m = cfac,
// i.e. per order m two GEMMs whose K axis is the ring pairs:
//     E[l, c] = sum_pairs p_l(x) Q+[pair, c]  (l - m even),  O likewise with Q-,
//     Q+- = q_N +- q_S  (columns c = 2 map + {re, im}).
// The cached tile of (m, ring block, stage) holds p_l for 128 pairs (rows of
// 32 bytes) x 16 degrees of one parity (K-major for the forward product).  A
// 1 KB slice of it (32 pairs) is exactly the MN-major 32-byte-swizzle layout
// of the transposed operand (M = degrees, K = pairs): 8 K rows of 32 bytes per
// 256-byte atom, atoms along K 256 bytes apart (stride byte offset), the next
// 16 degrees in the next stage's slice (leading byte offset 1 KB).  So the
// tensor core reads the forward's operand transposed, with no data movement
// other than the bulk copies of the slices.
constexpr int kAdjStages = 8;                 // stages per block of 128 degrees of one parity
constexpr int kAdjPairs = 32;                 // ring pairs per K chunk (two MMA K steps)
constexpr int kAdjSlice = kAdjPairs * kRowBytes;  // 1 KB
constexpr int kAdjWarps = 10;                 // 0-7 drain, 8 loads + tensor memory, 9 MMA

template <int NPA, int NPB>
struct AdjCfg {
    static constexpr int NS = 3;                                       // chunks in flight
    static constexpr int A_BYTES = 2 * NPA * kAdjStages * kAdjSlice;  // [par][piece][stage] slices
    static constexpr int B_MAX = 2 * NPB * 2 * 64 * kRowBytes;         // [par][piece][ksub] x N <= 64 rows
    static constexpr int STAGE_BYTES = A_BYTES + B_MAX;
    static constexpr int NPROD = (NPA == 2 && NPB == 2) ? 3 : 6;
    static constexpr int SMEM = NS * STAGE_BYTES + 1024 /* align */ + 256 /* barriers */;
};

// MN-major operand with the 32-byte swizzle: leading byte offset = stride of
// the 32-byte column blocks along M, stride byte offset = stride of the
// 8-row groups along K (descriptor version 1).
__device__ __forceinline__ uint64_t sdesc_sw32_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)6 << 61;
    return d;
}

// Operand image of the transpose: for every (m, chunk c of 32 pairs) a block
// of 2 x NPB x 2 tiles ([parity][piece][ksub], N rows of 32 bytes each, row n
// = 2 map + {re, im} holding 16 pairs, 16-byte halves swizzled by bit 2 of
// the row) of the pieces of Q+ (parity 0) and Q- (parity 1).  q is the FP32
// ring analysis [map][ring][m].  One thread per (m, map b < N / 2, c), m
// fastest so that the reads of q are coalesced; maps b >= nmaps and pairs past
// the last are zero.
template <int NPB>
__global__ void __launch_bounds__(256)
adj_prep_kernel(const DevPlan P, const float2 *__restrict__ q, unsigned char *__restrict__ bout, int nmaps, int ncol)
{
    const int M1 = P.mmax + 1;
    const int nch = (P.npairs + kAdjPairs - 1) / kAdjPairs;
    const int nb2 = ncol >> 1;
    const int c = blockIdx.y;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M1 * nb2) return;
    const int m = idx % M1, b = idx / M1;
    const size_t blk = (size_t)2 * NPB * 2 * ncol * kRowBytes;
    unsigned char *out = bout + ((size_t)m * nch + c) * blk;
    const float2 *qb = q + (size_t)b * P.nrings * M1 + m;
#pragma unroll 1
    for (int ks = 0; ks < 2; ++ks) {
        float2 e[16], o[16];
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const int pair = c * kAdjPairs + 16 * ks + kk;
            float2 vn = make_float2(0.f, 0.f), vs = make_float2(0.f, 0.f);
            if (pair < P.npairs && b < nmaps) {
                const int2 rr = P.pair_ring[pair];
                vn = qb[(size_t)rr.x * M1];
                if (rr.y >= 0) vs = qb[(size_t)rr.y * M1];
            }
            e[kk] = make_float2(vn.x + vs.x, vn.y + vs.y);
            o[kk] = make_float2(vn.x - vs.x, vn.y - vs.y);
        }
#pragma unroll
        for (int par = 0; par < 2; ++par) {
#pragma unroll
            for (int col = 0; col < 2; ++col) {
                const int n = 2 * b + col;
                uint32_t w[NPB][8];
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
                    const float2 v = par ? o[kk] : e[kk];
                    uint32_t pc[NPB];
                    split_pieces<true, NPB>(col ? v.y : v.x, pc);
#pragma unroll
                    for (int pq = 0; pq < NPB; ++pq) {
                        if (kk & 1)
                            w[pq][kk >> 1] |= pc[pq] & 0xFFFF0000u;
                        else
                            w[pq][kk >> 1] = pc[pq] >> 16;
                    }
                }
                const int sw = (n >> 2) & 1;
#pragma unroll
                for (int pq = 0; pq < NPB; ++pq) {
                    unsigned char *row = out + ((size_t)((par * NPB + pq) * 2 + ks) * ncol + n) * kRowBytes;
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        *reinterpret_cast<uint4 *>(row + ((h ^ sw) << 4)) =
                            make_uint4(w[pq][4 * h], w[pq][4 * h + 1], w[pq][4 * h + 2], w[pq][4 * h + 3]);
                }
            }
        }
    }
}

// Persistent, one CTA per SM over the items (m, block j of 128 degrees of
// each parity), taken round robin in increasing m; per item the K loop runs
// over the chunks of 32 ring pairs:
//   warps 0-7  drain: warp w reads tensor-memory lanes 32 (w % 4) .. + 32
//              (rows = degrees) of E (w < 4) or O; after every chunk it adds
//              the finished accumulator into its register totals (FP32, round
//              to nearest: the tensor core's truncating accumulation stays
//              within 12 MMAs, as in the forward kernels), and at the end
//              writes g_lm = c C_l (E or O) for its degrees and maps;
//   warp 8     tensor memory, and the chunk's copies: the block's stage
//              slices of the cached operand (1 KB each) and the chunk's
//              block of the transpose operand image, on one mbarrier;
//   warp 9     the MMAs: per parity, 2 K steps x the piece products, A
//              MN-major from the slices, B K-major; D alternates between two
//              accumulator sets per chunk.
// Chunks without a value in FP32 range are left out: past the order limit of
// their ring block, or all of the block's degrees before the block's first
// nonzero stage (evanescent skip).  Slices of stages past the order's last
// stage are not loaded: the rows they feed are degrees above lmax, which are
// never written.  Every wait is bounded as in the forward kernels.
template <int NPA, int NPB>
__global__ void __launch_bounds__(kAdjWarps * 32, 1)
legendre_adj_tc_kernel(const DevPlan P, const unsigned char *__restrict__ acache, const int *__restrict__ seg_off,
                       const unsigned char *__restrict__ bimg, const int2 *__restrict__ items, int nitems,
                       double2 *__restrict__ g, int nmaps, int ncol, double cfac, int *__restrict__ status,
                       const __grid_constant__ CUtensorMap amap, int use_tma)
{
    using A = AdjCfg<NPA, NPB>;
    constexpr int NS = A::NS;
    constexpr int STEPS = 32;               // degrees per cached stage (BF16)
    constexpr int GROUP = 64 / STEPS;       // stages per skip group
    constexpr size_t SA = (size_t)2 * NPA * kTileBytes;  // one cached stage block
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t base_u32 = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (base_u32 & 1023u)) & 1023u;
    unsigned char *stage0 = smem_raw + pad;
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage0 + NS * A::STAGE_BYTES);
    // bars: full[NS], empty[NS], set_full[2], set_empty[2], mma_drain
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int L = P.lmax;
    const int nrb = (P.npairs + kRows - 1) / kRows;
    const int nch = (P.npairs + kAdjPairs - 1) / kAdjPairs;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t sbb = (uint32_t)2 * NPB * 2 * ncol * kRowBytes;  // operand image block per chunk
    SHT_CHECK(P.dbg, (ncol == 32 || ncol == 64) && 2 * nmaps <= ncol, 501);
    // persistent: the CTA runs items blockIdx.x, + gridDim.x, ...; every role
    // walks the same sequence, and the barrier phases run on across items
    struct Item {
        int m, j, nst, i_lo, i_hi;  // order, degree block, stages of m, the block's cached stages
    };
    auto item_of = [&](int t) {
        const int2 it = items[t];
        Item I;
        I.m = it.x;
        I.j = it.y;
        I.nst = (L - I.m + 1 + STEPS - 1) / STEPS;
        I.i_lo = kAdjStages * I.j;
        I.i_hi = min(I.nst, I.i_lo + kAdjStages);
        return I;
    };

    auto bar_full = [&](int s) { return smem_u32(&bars[s]); };
    auto bar_empty = [&](int s) { return smem_u32(&bars[NS + s]); };
    auto bar_set_full = [&](int k) { return smem_u32(&bars[2 * NS + k]); };
    auto bar_set_empty = [&](int k) { return smem_u32(&bars[2 * NS + 2 + k]); };
    const uint32_t bar_mma_drain = smem_u32(&bars[2 * NS + 4]);
    // A slices of a chunk: [stage][parity][piece], 1 KB each (the order of a
    // tensor-map box over the cached operand), so consecutive 16-degree blocks
    // of one (parity, piece) are 2 NPA KB apart (the MN-major leading byte offset)
    constexpr uint32_t kLbo = 2 * NPA * kAdjSlice;
    auto a_slice = [&](int s, int par, int piece, int st) {
        return stage0 + (size_t)s * A::STAGE_BYTES + (size_t)(st * 2 * NPA + par * NPA + piece) * kAdjSlice;
    };
    auto b_tile = [&](int s, int par, int piece, int ks) {
        return stage0 + (size_t)s * A::STAGE_BYTES + A::A_BYTES + (size_t)((par * NPB + piece) * 2 + ks) * ncol * kRowBytes;
    };
    // chunk k (pairs 32 k ..) of ring block k / 4 runs iff it has pairs, the
    // block has a value in FP32 range at this order, and the item's degrees
    // reach the block's first nonzero stage
    auto live = [&](const Item &I, int k) {
        const int rb = k >> 2;
        if (P.block_mlim && I.m >= P.block_mlim[rb]) return false;
        const int s0 = P.skip_g ? P.skip_g[I.m * nrb + rb] * GROUP : 0;
        return I.i_hi > s0;
    };

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < NS; ++s) {
            mbar_init(bar_full(s), 1);
            mbar_init(bar_empty(s), 1);
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(bar_set_full(k), 1);
            mbar_init(bar_set_empty(k), 8);
        }
        mbar_init(bar_mma_drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(256u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp < 8) {
        // ----------------------------------------------------------- drain --
        const int quad = warp & 3;
        const int half = warp >> 2;  // 0: E (l - m even), 1: O
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        uint32_t gg = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
            const Item I = item_of(t);
            float tot[64];
#pragma unroll
            for (int c = 0; c < 64; ++c) tot[c] = 0.f;
            for (int k = 0; k < nch && ok; ++k) {
                if (!live(I, k)) continue;
                const int set = (int)(gg & 1u);
                ok = __all_sync(0xffffffffu, mbar_wait(bar_set_full(set), (gg >> 1) & 1u, &s_abort));
                if (!ok) break;
                tc_fence_after();
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (32 * h < ncol) {
                        uint32_t v[32];
                        tmem_ld32(tmem + lane_base + (uint32_t)(128 * set + half * ncol + 32 * h), v);
#pragma unroll
                        for (int c = 0; c < 32; ++c) tot[32 * h + c] += __uint_as_float(v[c]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_set_empty(set));
                ++gg;
            }
            if (!ok) break;
            // row r = 16 (stage in the block) + position in the stage's parity
            const int m = I.m;
            const int r = quad * 32 + lane;
            const int l = m + 2 * (kAdjStages * 16 * I.j + r) + half;
            if (l <= L) {
                const long long mofs = (long long)m * (2 * L + 3 - m) / 2;
                const double cl = (m == 0 ? 1.0 : cfac) * __ldg(&P.coefC[mofs + (l - m)]);
                double2 *dst = g + mofs + (l - m);
#pragma unroll
                for (int b = 0; b < 32; ++b)
                    if (b < nmaps)
                        dst[(size_t)b * P.nalm] =
                            make_double2(cl * (double)tot[2 * b], m == 0 ? 0.0 : cl * (double)tot[2 * b + 1]);
            }
        }
    } else if (warp == 8) {
        // ---------------------------------------------------------- loads --
        if (lane == 0) {
            uint32_t gs = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
                const Item I = item_of(t);
                const size_t st0 = (size_t)(seg_off[2 * I.m] / STEPS);  // stages of the orders below m
                SHT_CHECK(P.dbg, I.i_lo < I.i_hi, 503);
                for (int k = 0; k < nch && ok; ++k) {
                    if (!live(I, k)) continue;
                    const int s = (int)(gs % NS);
                    const uint32_t ph = (gs / NS) & 1u;
                    if (!mbar_wait(bar_empty(s), ph ^ 1u, &s_abort)) {
                        ok = false;
                        break;
                    }
                    const int rb = k >> 2, w = k & 3;
                    const size_t sg = st0 * nrb + (size_t)rb * I.nst + I.i_lo;  // first stage, whole-operand index
                    if (use_tma) {
                        // one box: 8 stages x 2 NPA tiles x the chunk's 1 KB slice (stages
                        // past the operand's end read as zeros, the rest feed rows above lmax)
                        mbar_expect_tx(bar_full(s), (uint32_t)(kAdjStages * 2 * NPA * kAdjSlice) + sbb);
                        SHT_CHECK(P.dbg, sg < 0x7fffffffull, 504);
                        asm volatile(
                            "cp.async.bulk.tensor.4d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
                                smem_u32(a_slice(s, 0, 0, 0))),
                            "l"(reinterpret_cast<uint64_t>(&amap)), "r"(0), "r"(w), "r"(0), "r"((int)sg),
                            "r"(bar_full(s))
                            : "memory");
                    } else {
                        mbar_expect_tx(bar_full(s), (uint32_t)((I.i_hi - I.i_lo) * 2 * NPA * kAdjSlice) + sbb);
                        const unsigned char *ablk = acache + sg * SA;
                        for (int i = 0; i < I.i_hi - I.i_lo; ++i)
#pragma unroll
                            for (int par = 0; par < 2; ++par)
#pragma unroll
                                for (int pc = 0; pc < NPA; ++pc)
                                    bulk_load(smem_u32(a_slice(s, par, pc, i)),
                                              ablk + (size_t)i * SA + (size_t)(par * NPA + pc) * kTileBytes +
                                                  (size_t)w * kAdjSlice,
                                              kAdjSlice, bar_full(s));
                    }
                    bulk_load(smem_u32(b_tile(s, 0, 0, 0)), bimg + ((size_t)I.m * nch + k) * sbb, sbb, bar_full(s));
                    ++gs;
                }
            }
            if (s_abort) {
                const uint32_t first = gs > (uint32_t)NS ? gs - NS : 0u;
                for (uint32_t q = first; q < gs; ++q) mbar_drain(bar_full((int)(q % NS)), (q / NS) & 1u);
            }
        }
    } else {
        // ----------------------------------------------------------- MMA --
        if (lane == 0) {
            const uint32_t id = idesc<true>(ncol) | (1u << 15);  // A MN-major
            uint32_t gs = 0;
            bool ok = true, issued = false;
            for (int t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
                const Item I = item_of(t);
                for (int k = 0; k < nch && ok; ++k) {
                    if (!live(I, k)) continue;
                    const int s = (int)(gs % NS);
                    const uint32_t ph = (gs / NS) & 1u;
                    const int set = (int)(gs & 1u);
                    if (!mbar_wait(bar_set_empty(set), ((gs >> 1) & 1u) ^ 1u, &s_abort) ||
                        !mbar_wait(bar_full(s), ph, &s_abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    SHT_CHECK(P.dbg, 128 * set + 2 * ncol <= 256 && s < NS, 502);
#pragma unroll
                    for (int par = 0; par < 2; ++par) {
                        const uint32_t d = tmem + (uint32_t)(128 * set + par * ncol);
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
                            for (int pr = 0; pr < A::NPROD; ++pr) {
                                int ia, ib;
                                product_pieces<NPA, NPB>(pr, ia, ib);
                                // K step ks: pairs 16 ks .. 16 ks + 15 = two 8-row groups further
                                const uint64_t ad =
                                    sdesc_sw32_mn(smem_u32(a_slice(s, par, ia, 0)) + 512u * ks, kLbo, 256u);
                                const uint64_t bd = sdesc_sw32(smem_u32(b_tile(s, par, ib, ks)));
                                tc_mma<true>(d, ad, bd, id, (ks > 0 || pr > 0) ? 1u : 0u);
                            }
                        }
                    }
                    issued = true;
                    tc_commit(bar_empty(s));
                    tc_commit(bar_set_full(set));
                    ++gs;
                }
            }
            if (!ok && issued) {
                tc_commit(bar_mma_drain);
                mbar_drain(bar_mma_drain, 0u);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u));
    }
    if (threadIdx.x == 0 && s_abort) atomicExch(status, SHT_ETIMEOUT);
}

}  // namespace

cudaError_t launch_tc_main_multi(const DevPlan &P, const DevPlan *plans_dev, const int4 *items, int nitems,
                                 const MultiTcPtrs &mp, int prec, int *status, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    if (prec == SHT_FP32_TC) return run_main_multi<false, 2, 2>(P, plans_dev, items, nitems, mp, status, st);
    if (prec == SHT_BF16X3_TC) return run_main_multi<true, 2, 2>(P, plans_dev, items, nitems, mp, status, st);
    return run_main_multi<true, 3, 3>(P, plans_dev, items, nitems, mp, status, st);
}

size_t tc_bbuf_bytes(const TcWork &W, int prec)
{
    // pieces x 128 columns (the widest launch group) x K
    if (prec == SHT_FP32_TC) return (size_t)2 * 128 * W.kall_tf32 * 4;
    if (prec == SHT_BF16X3_TC) return (size_t)2 * 128 * W.kall_bf16 * 2;
    return (size_t)3 * 128 * W.kall_bf16 * 2;
}

size_t tc_lambda_bytes(const DevPlan &P, const TcWork &W, int prec)
{
    // stages of all orders x ring blocks x (2 parities x pieces x 4 KB)
    const size_t nrb = (size_t)((P.npairs + kRows - 1) / kRows);
    if (prec == SHT_FP32_TC) return (size_t)(W.kall_tf32 / 16) * nrb * 2 * 2 * kTileBytes;
    if (prec == SHT_BF16X3_TC) return (size_t)(W.kall_bf16 / 32) * nrb * 2 * 2 * kTileBytes;
    if (prec == SHT_BF16X6_TC) return (size_t)(W.kall_bf16 / 32) * nrb * 2 * 3 * kTileBytes;
    return 0;
}

size_t adj_tc_bimg_bytes(const DevPlan &P, int prec, int nmaps)
{
    const int npb = prec == SHT_BF16X6_TC ? 3 : 2;
    const int ncol = nmaps <= 16 ? 32 : 64;
    const size_t nch = (size_t)((P.npairs + kAdjPairs - 1) / kAdjPairs);
    return nch * (size_t)(P.mmax + 1) * 2 * npb * 2 * ncol * kRowBytes;
}

cudaError_t launch_adj_tc(const DevPlan &P, const TcWork &W, int prec, const void *acache, const float2 *q,
                          void *bimg, const int2 *items, int nitems, double2 *g, int nmaps, double cfac,
                          cudaStream_t st)
{
    if (nmaps <= 0 || nitems <= 0) return cudaSuccess;
    if (nmaps > 32 || (prec != SHT_BF16X3_TC && prec != SHT_BF16X6_TC)) return cudaErrorInvalidValue;
    const int ncol = nmaps <= 16 ? 32 : 64;
    const int nch = (P.npairs + kAdjPairs - 1) / kAdjPairs;
    dim3 pg(((P.mmax + 1) * (ncol >> 1) + 255) / 256, nch);
    unsigned char *bo = static_cast<unsigned char *>(bimg);
    const unsigned char *ac = static_cast<const unsigned char *>(acache);
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = std::min(nitems, std::max(1, nsm));  // persistent: one CTA per SM
    // the cached operand as a 4-D array of 32-bit words: (256 words = one 1 KB
    // slice of 32 pairs) x (4 slices of a tile) x (2 NPA tiles of a stage) x
    // stages; a box of 8 stages x 2 NPA tiles x 1 slice is one chunk's A
    CUtensorMap amap;
    std::memset(&amap, 0, sizeof amap);
    int use_tma = 0;
    {
        const int npa = prec == SHT_BF16X6_TC ? 3 : 2;
        const size_t sa = (size_t)2 * npa * kTileBytes;
        const size_t nstg = tc_lambda_bytes(P, W, prec) / sa;
        auto enc = tensor_map_encoder();
        if (enc && (reinterpret_cast<uintptr_t>(acache) & 15) == 0 && nstg > 0 && nstg < 0x7fffffffull) {
            const cuuint64_t dims[4] = {256, 4, (cuuint64_t)(2 * npa), (cuuint64_t)nstg};
            const cuuint64_t strides[3] = {(cuuint64_t)kAdjSlice, (cuuint64_t)kTileBytes, (cuuint64_t)sa};
            const cuuint32_t box[4] = {256, 1, (cuuint32_t)(2 * npa), (cuuint32_t)kAdjStages};
            const cuuint32_t es[4] = {1, 1, 1, 1};
            const CUresult cr = enc(&amap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, const_cast<void *>(acache), dims, strides,
                                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            use_tma = cr == CUDA_SUCCESS ? 1 : 0;
        }
    }
    if (prec == SHT_BF16X6_TC) {
        adj_prep_kernel<3><<<pg, 256, 0, st>>>(P, q, bo, nmaps, ncol);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        auto kern = legendre_adj_tc_kernel<3, 3>;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, AdjCfg<3, 3>::SMEM)) !=
            cudaSuccess)
            return e;
        kern<<<grid, kAdjWarps * 32, AdjCfg<3, 3>::SMEM, st>>>(P, ac, W.seg_bf16, bo, items, nitems, g, nmaps, ncol,
                                                                 cfac, W.status, amap, use_tma);
    } else {
        adj_prep_kernel<2><<<pg, 256, 0, st>>>(P, q, bo, nmaps, ncol);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        auto kern = legendre_adj_tc_kernel<2, 2>;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, AdjCfg<2, 2>::SMEM)) !=
            cudaSuccess)
            return e;
        kern<<<grid, kAdjWarps * 32, AdjCfg<2, 2>::SMEM, st>>>(P, ac, W.seg_bf16, bo, items, nitems, g, nmaps, ncol,
                                                                 cfac, W.status, amap, use_tma);
    }
    return cudaGetLastError();
}

cudaError_t launch_warm_start(const DevPlan &P, int *skip_g, double *warm_p0, double *warm_p1, int *warm_k,
                              int *pair_lim, cudaStream_t st)
{
    dim3 grid((P.npairs + kRows - 1) / kRows, P.mmax + 1);
    warm_start_kernel<<<grid, kRows, 0, st>>>(P, skip_g, warm_p0, warm_p1, warm_k, pair_lim);
    return cudaGetLastError();
}

cudaError_t launch_lambda_build(const DevPlan &P, const TcWork &W, int prec, void *out, cudaStream_t st)
{
    dim3 grid((P.npairs + kRows - 1) / kRows, P.mmax + 1);
    unsigned char *o = static_cast<unsigned char *>(out);
    if (prec == SHT_FP32_TC)
        lambda_build_kernel<false, 2><<<grid, kRows, 0, st>>>(P, W.seg_tf32, o);
    else if (prec == SHT_BF16X3_TC)
        lambda_build_kernel<true, 2><<<grid, kRows, 0, st>>>(P, W.seg_bf16, o);
    else if (prec == SHT_BF16X6_TC)
        lambda_build_kernel<true, 3><<<grid, kRows, 0, st>>>(P, W.seg_bf16, o);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_tc_prep(const DevPlan &P, const TcWork &W, int prec, const double2 *alm, int nmaps, cudaStream_t st)
{
    if (nmaps <= 0) return cudaSuccess;
    if (nmaps > kTcMaxMaps) return cudaErrorInvalidValue;
    if (prec == SHT_FP32_TC) return run_prep<false, 2, 2>(P, W, alm, nmaps, st);
    if (prec == SHT_BF16X3_TC) return run_prep<true, 2, 2>(P, W, alm, nmaps, st);
    return run_prep<true, 3, 3>(P, W, alm, nmaps, st);
}

cudaError_t launch_tc_prep_multi(const DevPlan *plans_dev, const int2 *items, int nitems, const MultiTcPtrs &mp,
                                 int prec, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    if (prec == SHT_FP32_TC)
        prep_b_multi_kernel<false, 2><<<nitems, 256, 0, st>>>(plans_dev, items, mp);
    else if (prec == SHT_BF16X3_TC)
        prep_b_multi_kernel<true, 2><<<nitems, 256, 0, st>>>(plans_dev, items, mp);
    else
        prep_b_multi_kernel<true, 3><<<nitems, 256, 0, st>>>(plans_dev, items, mp);
    return cudaGetLastError();
}

cudaError_t launch_tc_main(const DevPlan &P, const TcWork &W, int prec, const void *acache, float2 *delta, int nmaps,
                           cudaStream_t st)
{
    if (nmaps <= 0) return cudaSuccess;
    if (nmaps > kTcMaxMaps) return cudaErrorInvalidValue;
    if (prec == SHT_FP32_TC) return run_main<false, 2, 2>(P, W, acache, delta, nmaps, st);
    if (prec == SHT_BF16X3_TC) return run_main<true, 2, 2>(P, W, acache, delta, nmaps, st);
    return run_main<true, 3, 3>(P, W, acache, delta, nmaps, st);
}

}  // namespace sht
