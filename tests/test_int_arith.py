"""The integer-pipe arithmetic of the tensor-core producer, on the host: the
helpers of csrc/legendre_tc.cu are compiled as they stand with g++ (CUDA
intrinsics replaced by host equivalents) and checked against IEEE-754.

- mul_coef (the coefficient product A x on the integer pipes) must equal the
  correctly rounded product, fma(A, x, +0), bit for bit, including exact ties
  (A with a short significand such as 3 or 1.5) and x = 0;
- rn_f32 (FP64 -> FP32 on the integer pipe) must round to nearest with ties
  away from zero, and flush values below the FP32 normal range to signed zero;
- split_pieces (the operand pieces of the tensor-core forms) must leave exact
  residuals and rounded (not truncated) pieces, each later piece at most half
  an ulp of the one before (|lo| <= 2^-11 |v| for TF32; |mid| <= 2^-8 |v|,
  |lo| <= 2^-16 |v| for BF16): the bounds on the products the forms leave
  out.  2 TF32 pieces rebuild the value to 2^-23 relative, 3 BF16 pieces
  exactly (24 bits), both floored at 2^-126 below the FP32 normal range.
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1010_1260_gb300", "csrc", "legendre_tc.cu")
OUT = os.path.join(ROOT, "paper_1010_1260_gb300", "_build")

SHIM = r"""
#include <cstdint>
#include <cstring>
#include <cmath>
#include <cstdio>
static inline long long __double_as_longlong(double d) { long long r; std::memcpy(&r, &d, 8); return r; }
static inline double __longlong_as_double(long long u) { double d; std::memcpy(&d, &u, 8); return d; }
static inline int __double2hiint(double d) { return (int)(__double_as_longlong(d) >> 32); }
static inline int __double2loint(double d) { return (int)(unsigned)__double_as_longlong(d); }
static inline float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static inline unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static inline unsigned long long __umul64hi(unsigned long long a, unsigned long long b)
{ return (unsigned long long)(((unsigned __int128)a * b) >> 64); }
static inline unsigned __funnelshift_r(unsigned lo, unsigned hi, unsigned s)
{ return (unsigned)((((unsigned long long)hi << 32) | lo) >> (s & 31)); }
"""

DRIVER = r"""
static uint64_t s_ = 0x9E3779B97F4A7C15ull;
static uint64_t nxt() { s_ ^= s_ << 13; s_ ^= s_ >> 7; s_ ^= s_ << 17; return s_; }
static double uni() { return (double)(nxt() >> 11) * 0x1p-53; }
int main() {
    long bad_mul = 0, bad_rn = 0, n_mul = 0, n_rn = 0;
    // coefficient products: generic, short significands (exact ties), zeros, x < 0, tiny x
    for (long i = 0; i < 3000000; ++i) {
        double a;
        switch (i % 4) {
            case 0: a = (double)(1 + i % 97); break;                     // integers: short significands
            case 1: a = 1.5 * std::ldexp(1.0, (int)(i % 7)) + 0.25 * (i % 5); break;
            case 2: a = std::sqrt((double)(2 * (i % 2000) + 3)); break;  // sqrt(2m+3), some exact
            default: a = 0.01 + 70.0 * uni();
        }
        if (i % 101 == 0) a = 0.0;
        double x = (i % 5 == 0) ? (double)(2 * (i % 61) + 1) / 128.0 : uni();
        if (i % 13 == 0) x = 0.0;
        if (i % 17 == 0) x = -x;
        if (i % 19 == 0) x = std::ldexp(uni() + 0.5, -40);
        const double want = std::fma(a, x, 0.0);
        const double got = sht::mul_coef(a, sht::xint_of(x));
        ++n_mul;
        if (std::memcmp(&want, &got, 8) != 0 && ++bad_mul <= 3)
            std::printf("mul_coef(%a, %a) = %a, want %a\n", a, x, got, want);
    }
    // FP64 -> FP32: every exponent of the domain (|d| < 2^128), both signs, rounding edges
    for (int e = 0; e <= 1023 + 127; ++e) {
        for (int k = 0; k < 4000; ++k) {
            uint64_t m = nxt() & 0xFFFFFFFFFFFFFull;
            if (k < 4) m = (k & 1) ? 0 : 0xFFFFFFFFFFFFFull;
            else if (k < 12) m = (m & ~0x1FFFFFFFull) | ((uint64_t)(k & 1) << 28);  // exact halves
            const uint64_t u = ((nxt() >> 63) << 63) | ((uint64_t)e << 52) | m;
            const double d = __longlong_as_double((long long)u);
            const float got = sht::rn_f32(d);
            float want;
            const double ad = std::fabs(d);
            if (ad < 0x1p-126) {
                want = std::signbit(d) ? -0.0f : 0.0f;
            } else {
                const float t = (float)ad;  // round to nearest even (host default)
                const float lo = ((double)t > ad) ? std::nextafterf(t, 0.0f) : t;
                const float hi = std::nextafterf(lo, INFINITY);
                const double hv = std::isinf(hi) ? 0x1p128 : (double)hi;  // above FLT_MAX: 2^128 (inf)
                const double dl = ad - (double)lo, dh = hv - ad;
                const float r = (dl < dh) ? lo : (dh < dl) ? hi : hi;   // ties away from zero
                want = std::signbit(d) ? -r : r;
            }
            ++n_rn;
            if (std::memcmp(&want, &got, 4) != 0 && ++bad_rn <= 3)
                std::printf("rn_f32(%a) = %a, want %a\n", d, (double)got, (double)want);
        }
    }
    // operand pieces: exact residuals and the reconstruction bounds
    long bad_split = 0, n_split = 0;
    for (long i = 0; i < 2000000; ++i) {
        const float v = (float)((uni() - 0.5) * std::ldexp(1.0, (int)(nxt() % 200) - 100));
        if (v == 0.0f) continue;
        uint32_t t[2], b[3];
        sht::split_pieces<false, 2>(v, t);
        sht::split_pieces<true, 3>(v, b);
        double rt = v, rb = v;
        bool ok = true;
        for (int q = 0; q < 2; ++q) {
            const double pq = __uint_as_float(t[q]);
            ok = ok && ((t[q] & 0x1FFFu) == 0u);                       // a TF32 value
            ok = ok && ((double)(float)(rt - pq) == rt - pq);          // exact residual
            rt -= pq;
        }
        for (int q = 0; q < 3; ++q) {
            const double pq = __uint_as_float(b[q] & 0xFFFF0000u);
            ok = ok && ((double)(float)(rb - pq) == rb - pq);
            rb -= pq;
        }
        const double av = std::fabs((double)v);
        const double t1 = std::fabs((double)__uint_as_float(t[1]));
        const double b1 = std::fabs((double)__uint_as_float(b[1] & 0xFFFF0000u));
        const double b2 = std::fabs((double)__uint_as_float(b[2] & 0xFFFF0000u));
        if (av >= 0x1p-100) {
            // rounded (not truncated) pieces: each later piece at most half an ulp
            // of the one before; 3 BF16 pieces hold all 24 bits of an FP32 value
            ok = ok && t1 <= 0x1.02p-11 * av && std::fabs(rt) <= std::ldexp(av, -23);
            ok = ok && b1 <= 0x1.02p-8 * av && b2 <= 0x1.04p-16 * av && rb == 0.0;
        } else {
            // later pieces may fall below the FP32 normal range: the relative
            // bounds, floored at its minimum
            ok = ok && std::fabs(rt) <= std::fmax(std::ldexp(av, -23), 0x1p-126);
            ok = ok && std::fabs(rb) <= 0x1p-126;
        }
        ++n_split;
        if (!ok && ++bad_split <= 3)
            std::printf("split_pieces(%a): residuals %a (tf32x2) %a (bf16x3)\n", (double)v, rt, rb);
    }
    std::printf("mul_coef %ld/%ld bad, rn_f32 %ld/%ld bad, split %ld/%ld bad\n", bad_mul, n_mul, bad_rn, n_rn,
                bad_split, n_split);
    return (bad_mul || bad_rn || bad_split) ? 1 : 0;
}
"""


def _extract(src: str, start: str, end: str) -> str:
    i = src.index(start)
    return src[i:src.index(end, i)]


@pytest.fixture(scope="module")
def program():
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    src = open(SRC).read()
    parts = [_extract(src, "__device__ __forceinline__ float rn_f32(double d)",
                      "// The coefficient product A_l x of the recurrence"),
             _extract(src, "struct XInt {", "// degrees (by position in the stage)")]
    body = "\n".join(parts)
    body = re.sub(r"__device__\s+__forceinline__", "static inline", body)
    code = SHIM + "namespace sht {\n" + body + "\n}\n" + DRIVER
    os.makedirs(OUT, exist_ok=True)
    cpp = os.path.join(OUT, "int_arith_check.cpp")
    exe = os.path.join(OUT, "int_arith_check")
    with open(cpp, "w") as f:
        f.write(code)
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe, cpp],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def test_integer_product_and_rounding_match_ieee(program):
    r = subprocess.run([program], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:]
    assert "mul_coef 0/" in r.stdout and "rn_f32 0/" in r.stdout and "split 0/" in r.stdout
