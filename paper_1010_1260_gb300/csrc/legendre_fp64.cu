// Legendre step in FP64: Delta_m(theta_r) = sum_{l >= m} a_lm lambda_lm(cos theta_r)
// (Eq. DeltaDef) for every order m and ring r.
//
// Mapping (GB300): one CTA per (ring-pair block of 128, m, map group).  Each
// thread owns one pair of mirrored rings and walks l = m..lmax sequentially
// (the recurrence of Eq. assLegRec is serial in l).  The per-l data shared by
// the CTA -- the recurrence coefficient A_{l+1} and the prescaled
// coefficients C_l a_lm of the CTA's maps -- is staged through shared memory
// in chunks of 64 l with coalesced loads and read back as broadcasts.
//
// Recurrence form.  With lambda_l = C_l p_l, C_m = C_{m+1} = 1 and
// C_l = (beta_l / beta_{l-1}) C_{l-2}, the normalised recurrence
//     lambda_l = beta_l (x lambda_{l-1} - lambda_{l-2} / beta_{l-1})
// becomes p_l = A_l x p_{l-1} - p_{l-2} with A_l = beta_{l-1} C_{l-1} / C_{l-2}
// (A_{m+1} = sqrt(2m+3), Eq. pm1m): one multiply and one FMA per step.
//
// North/south symmetry (sec. 2.2.1): lambda_lm(-x) = (-1)^(l-m) lambda_lm(x),
// so the even-(l-m) and odd-(l-m) partial sums E, O of the northern ring give
// Delta_m(north) = E + O and Delta_m(south) = E - O.
//
// Exponent tracking (Algorithm 2): the start value lambda_mm comes with an
// exponent k <= 0 (value = p * 2^(512 k)); while k < 0 the thread rescales
// when |p| > 2^256 and contributes nothing (the true value is < 2^-256).
#include "sht_internal.cuh"

#include <algorithm>
#include <type_traits>

namespace sht {
namespace {

constexpr int kThreads = 128;
constexpr int kChunk = 64;  // even, so every chunk starts on an even (l - m)

__device__ __forceinline__ bool above_hi(double v)
{
    // |v| > 2^kScaleHi, tested on the exponent bits (integer pipe)
    const int e = (__double2hiint(v) >> 20) & 0x7ff;
    return e > 1023 + kScaleHi;
}

// One work item: order m, ring pairs [pair_block * 128, + 128), maps [b0, b0 + BC).
// Every thread of the CTA must call it (it synchronises the CTA).
// Where an item writes: Delta of ring r, map b at delta[row_off[r] + b bstride
// + col] (row_off == nullptr: the full layout [map][ring][m], col = m).
struct OutMap {
    const long long *row_off = nullptr;
    long long bstride = 0;
    int col = 0;
};

template <int BC>
__device__ __forceinline__ void legendre_item(const DevPlan &P, const double2 *__restrict__ alm,
                                              double2 *__restrict__ delta, int nmaps, int m, int pair_block,
                                              int b0, double *sA, double2 (*sa)[BC], const OutMap &om = OutMap())
{
    const int L = P.lmax;
    const int pair = pair_block * kThreads + threadIdx.x;
    const bool live = pair < P.npairs;

    double x = 0.0, p0 = 0.0, p1 = 0.0;
    int k = 0;
    if (live) {
        const size_t so = SHT_IDX(P.dbg, (size_t)m * P.npairs + pair, (size_t)(P.mmax + 1) * P.npairs, 101);
        x = P.pair_x[pair];
        p1 = P.start_v[so];
        k = P.start_k[so];
    }
    double er[BC], ei[BC], orr[BC], oi[BC];
#pragma unroll
    for (int b = 0; b < BC; ++b) er[b] = ei[b] = orr[b] = oi[b] = 0.0;

    const long long mofs = (long long)m * (2 * L + 3 - m) / 2;  // packed index of (m, m)

    for (int l0 = m; l0 <= L; l0 += kChunk) {
        const int cnt = min(kChunk, L + 1 - l0);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += kThreads) {
            const int l = l0 + i;
            sA[i] = (l + 1 <= L) ? P.coefA[mofs + (l + 1 - m)] : 0.0;
        }
        for (int i = threadIdx.x; i < cnt * BC; i += kThreads) {
            const int b = i / cnt;
            const int j = i - b * cnt;
            const long long q = mofs + (l0 - m) + j;
            const double c = P.coefC[q];
            double2 a = make_double2(0.0, 0.0);
            if (b0 + b < nmaps) a = alm[SHT_IDX(P.dbg, (size_t)(b0 + b) * P.nalm + q, (size_t)nmaps * P.nalm, 102)];
            if (m == 0) a.y = 0.0;  // real field: Im(a_l0) is ignored
            sa[j][b] = make_double2(c * a.x, c * a.y);
        }
        __syncthreads();

        const bool slow = __any_sync(0xffffffffu, k < 0);
        if (!slow) {
            int j = 0;
            for (; j + 1 < cnt; j += 2) {
                // even (l - m): E
#pragma unroll
                for (int b = 0; b < BC; ++b) {
                    er[b] = fma(p1, sa[j][b].x, er[b]);
                    ei[b] = fma(p1, sa[j][b].y, ei[b]);
                }
                double t = fma(sA[j] * x, p1, -p0);
                p0 = p1;
                p1 = t;
                // odd (l - m): O
#pragma unroll
                for (int b = 0; b < BC; ++b) {
                    orr[b] = fma(p1, sa[j + 1][b].x, orr[b]);
                    oi[b] = fma(p1, sa[j + 1][b].y, oi[b]);
                }
                t = fma(sA[j + 1] * x, p1, -p0);
                p0 = p1;
                p1 = t;
            }
            if (j < cnt) {  // last l of the band, even (l - m)
#pragma unroll
                for (int b = 0; b < BC; ++b) {
                    er[b] = fma(p1, sa[j][b].x, er[b]);
                    ei[b] = fma(p1, sa[j][b].y, ei[b]);
                }
                const double t = fma(sA[j] * x, p1, -p0);
                p0 = p1;
                p1 = t;
            }
        } else {
            for (int j = 0; j < cnt; ++j) {
                if (k == 0) {
                    if ((j & 1) == 0) {
#pragma unroll
                        for (int b = 0; b < BC; ++b) {
                            er[b] = fma(p1, sa[j][b].x, er[b]);
                            ei[b] = fma(p1, sa[j][b].y, ei[b]);
                        }
                    } else {
#pragma unroll
                        for (int b = 0; b < BC; ++b) {
                            orr[b] = fma(p1, sa[j][b].x, orr[b]);
                            oi[b] = fma(p1, sa[j][b].y, oi[b]);
                        }
                    }
                }
                const double t = fma(sA[j] * x, p1, -p0);
                p0 = p1;
                p1 = t;
                if (k < 0 && above_hi(p1)) {
                    p1 *= 0x1p-512;
                    p0 *= 0x1p-512;
                    k += 1;
                }
            }
        }
    }

    if (!live) return;
    const int2 rr = P.pair_ring[pair];
    const int M1 = P.mmax + 1;
    if (om.row_off) {
#pragma unroll
        for (int b = 0; b < BC; ++b) {
            if (b0 + b >= nmaps) break;
            const long long o = (long long)(b0 + b) * om.bstride + om.col;
            const long long tot = (long long)P.nrings * nmaps * om.bstride;
            delta[SHT_IDX(P.dbg, om.row_off[rr.x] + o, tot, 103)] = make_double2(er[b] + orr[b], ei[b] + oi[b]);
            if (rr.y >= 0)
                delta[SHT_IDX(P.dbg, om.row_off[rr.y] + o, tot, 103)] = make_double2(er[b] - orr[b], ei[b] - oi[b]);
        }
        return;
    }
#pragma unroll
    for (int b = 0; b < BC; ++b) {
        if (b0 + b >= nmaps) break;
        const size_t tot = (size_t)nmaps * P.nrings * M1, o = (size_t)(b0 + b) * P.nrings * M1;
        delta[SHT_IDX(P.dbg, o + (size_t)rr.x * M1 + m, tot, 104)] = make_double2(er[b] + orr[b], ei[b] + oi[b]);
        if (rr.y >= 0)
            delta[SHT_IDX(P.dbg, o + (size_t)rr.y * M1 + m, tot, 104)] = make_double2(er[b] - orr[b], ei[b] - oi[b]);
    }
}

template <int BC>
__global__ void __launch_bounds__(kThreads)
legendre_fwd_fp64_kernel(const __grid_constant__ DevPlan P, const double2 *__restrict__ alm,
                         double2 *__restrict__ delta, int nmaps)
{
    __shared__ double sA[kChunk];        // A_{l+1} for l in the chunk
    __shared__ double2 sa[kChunk][BC];   // C_l a_lm for the CTA's maps
    legendre_item<BC>(P, alm, delta, nmaps, blockIdx.y, blockIdx.x, blockIdx.z * BC, sA, sa);
}

// ---------------------------------------------------------------- spin 2 --
// Polarisation (spin-2) Legendre step, FP64: for E/B coefficients the Q and U
// maps are two ordinary real syntheses (Eq. Delta2map) of
//   DQ_m = -sum_l (E_lm F1_lm + i B_lm F2_lm),  DU_m = -sum_l (B_lm F1_lm - i E_lm F2_lm),
// with F1 = (2lambda + -2lambda)/2 and F2 = (2lambda - -2lambda)/2 of the
// spin-weighted functions 2Y_lm = ð ð Y_lm / K_l, -2Y_lm = ð̄ ð̄ Y_lm / K_l,
// K_l = sqrt((l-1) l (l+1) (l+2)).  Eliminating the derivatives with the
// Legendre equation and sin t dlambda_l/dt = l c lambda_l - c_lm lambda_{l-1},
// c_lm = sqrt((2l+1)(l^2-m^2)/(2l-1)), with lambda_l = C_l p_l (the scaled
// recurrence), c = cos t and u = 1/sin^2 t:
//   K F1 = C_l p_l (2 m^2 u - 2 l c^2 u - l(l+1)) + 2 c u c_lm C_{l-1} p_{l-1},
//   K F2 = 2 m u ((1-l) c C_l p_l + c_lm C_{l-1} p_{l-1}).
// With X~ = X C_l / K_l and X^ = X c_lm C_{l-1} / K_l staged per degree, the
// thread keeps four sums per field and parity of l - m,
//   T0 = sum X~ p_l, T1 = sum l X~ p_l, T2 = sum l(l+1) X~ p_l, T3 = sum X^ p_{l-1},
// and the ring factors come after the sums:
//   sum X F1 = 2 m^2 u T0 - 2 c^2 u T1 - T2 + 2 c u T3,  sum X F2 = 2 m u (c (T0 - T1) + T3).
// North/south (lambda_lm(-x) = (-1)^(l-m) lambda_lm(x)): F1 of the southern
// ring takes T = T_even - T_odd, F2 the negative of that (its parity is
// opposite), both with the northern ring's c.  Output: Delta of component q
// (0: Q, 1: U) of map b at delta[((2 b + q) nrings + ring) (mmax+1) + m].
template <int BC>
__device__ __forceinline__ void legendre_spin2_item(const DevPlan &P, const double2 *__restrict__ elm,
                                                    const double2 *__restrict__ blm, double2 *__restrict__ delta,
                                                    int nmaps, int m, int pair_block, int b0, double *sA,
                                                    double2 (*sx)[BC][4])
{
    const int L = P.lmax;
    const int pair = pair_block * kThreads + threadIdx.x;
    const bool live = pair < P.npairs;
    double x = 0.0, p0 = 0.0, p1 = 0.0;
    int k = 0;
    if (live) {
        const size_t so = SHT_IDX(P.dbg, (size_t)m * P.npairs + pair, (size_t)(P.mmax + 1) * P.npairs, 105);
        x = P.pair_x[pair];
        p1 = P.start_v[so];
        k = P.start_k[so];
    }
    // T[b][field][sum][parity] as (re, im)
    double tr[BC][2][4][2], ti[BC][2][4][2];
#pragma unroll
    for (int b = 0; b < BC; ++b)
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
            for (int q = 0; q < 4; ++q) tr[b][f][q][0] = tr[b][f][q][1] = ti[b][f][q][0] = ti[b][f][q][1] = 0.0;
    const long long mofs = (long long)m * (2 * L + 3 - m) / 2;
    for (int l0 = m; l0 <= L; l0 += kChunk) {
        const int cnt = min(kChunk, L + 1 - l0);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += kThreads) {
            const int l = l0 + i;
            sA[i] = (l + 1 <= L) ? P.coefA[mofs + (l + 1 - m)] : 0.0;
        }
        for (int i = threadIdx.x; i < cnt * BC; i += kThreads) {
            const int b = i / cnt;
            const int j = i - b * cnt;
            const int l = l0 + j;
            const long long q = mofs + (l0 - m) + j;
            double2 e = make_double2(0.0, 0.0), bb = make_double2(0.0, 0.0);
            if (b0 + b < nmaps) {
                const size_t ai = SHT_IDX(P.dbg, (size_t)(b0 + b) * P.nalm + q, (size_t)nmaps * P.nalm, 106);
                e = elm[ai];
                bb = blm[ai];
            }
            if (m == 0) e.y = bb.y = 0.0;  // real fields: E_l0, B_l0 real
            double ct = 0.0, ch = 0.0;      // C_l / K_l and c_lm C_{l-1} / K_l (0 below l = 2)
            if (l >= 2) {
                const double dl = l, dm = m;
                const double K = sqrt((dl - 1.0) * dl * (dl + 1.0) * (dl + 2.0));
                ct = P.coefC[q] / K;
                if (l > m) ch = sqrt((2.0 * dl + 1.0) * (dl * dl - dm * dm) / (2.0 * dl - 1.0)) * P.coefC[q - 1] / K;
            }
            sx[j][b][0] = make_double2(ct * e.x, ct * e.y);
            sx[j][b][1] = make_double2(ch * e.x, ch * e.y);
            sx[j][b][2] = make_double2(ct * bb.x, ct * bb.y);
            sx[j][b][3] = make_double2(ch * bb.x, ch * bb.y);
        }
        __syncthreads();
        // one degree: contributions (while k == 0) to the sums of parity PAR of
        // l - m (chunks start on even l - m), then one recurrence step
        auto step = [&](int j, auto par_c) {
            constexpr int par = decltype(par_c)::value;
            if (k == 0) {
                const double dl = l0 + j, dll = dl * (dl + 1.0);
#pragma unroll
                for (int b = 0; b < BC; ++b)
#pragma unroll
                    for (int f = 0; f < 2; ++f) {
                        const double2 xt = sx[j][b][2 * f], xh = sx[j][b][2 * f + 1];
                        const double t_r = xt.x * p1, t_i = xt.y * p1;
                        tr[b][f][0][par] += t_r;
                        ti[b][f][0][par] += t_i;
                        tr[b][f][1][par] = fma(dl, t_r, tr[b][f][1][par]);
                        ti[b][f][1][par] = fma(dl, t_i, ti[b][f][1][par]);
                        tr[b][f][2][par] = fma(dll, t_r, tr[b][f][2][par]);
                        ti[b][f][2][par] = fma(dll, t_i, ti[b][f][2][par]);
                        tr[b][f][3][par] = fma(xh.x, p0, tr[b][f][3][par]);
                        ti[b][f][3][par] = fma(xh.y, p0, ti[b][f][3][par]);
                    }
            }
            const double t = fma(sA[j] * x, p1, -p0);
            p0 = p1;
            p1 = t;
            if (k < 0 && above_hi(p1)) {
                p1 *= 0x1p-512;
                p0 *= 0x1p-512;
                k += 1;
            }
        };
        for (int j = 0; j < cnt; j += 2) {
            step(j, std::integral_constant<int, 0>());
            if (j + 1 < cnt) step(j + 1, std::integral_constant<int, 1>());
        }
    }
    if (!live) return;
    const int2 rr = P.pair_ring[pair];
    const int M1 = P.mmax + 1;
    const double c = x, u = 1.0 / ((1.0 - x) * (1.0 + x));
    const double dm = m;
#pragma unroll
    for (int b = 0; b < BC; ++b) {
        if (b0 + b >= nmaps) break;
        // sum X F1 and sum X F2 of field f (0: E, 1: B) for the sign sg of the odd sums
        auto sums = [&](int f, double sg, double &f1r, double &f1i, double &f2r, double &f2i) {
            double T[4][2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                T[q][0] = tr[b][f][q][0] + sg * tr[b][f][q][1];
                T[q][1] = ti[b][f][q][0] + sg * ti[b][f][q][1];
            }
#pragma unroll
            for (int z = 0; z < 2; ++z) {
                const double v1 = 2.0 * dm * dm * u * T[0][z] - 2.0 * c * c * u * T[1][z] - T[2][z] + 2.0 * c * u * T[3][z];
                const double v2 = 2.0 * dm * u * (c * (T[0][z] - T[1][z]) + T[3][z]);
                if (z == 0) {
                    f1r = v1;
                    f2r = v2;
                } else {
                    f1i = v1;
                    f2i = v2;
                }
            }
        };
        const int rings[2] = {rr.x, rr.y};
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int ring = rings[side];
            if (ring < 0) continue;
            const double sg = side == 0 ? 1.0 : -1.0;
            double e1r, e1i, e2r, e2i, b1r, b1i, b2r, b2i;
            sums(0, sg, e1r, e1i, e2r, e2i);
            sums(1, sg, b1r, b1i, b2r, b2i);
            if (side == 1) {  // F2 of the southern ring has the opposite parity
                e2r = -e2r;
                e2i = -e2i;
                b2r = -b2r;
                b2i = -b2i;
            }
            // DQ = -(E F1 + i B F2), DU = -(B F1 - i E F2)
            const double2 dq = make_double2(-(e1r - b2i), -(e1i + b2r));
            const double2 du = make_double2(-(b1r + e2i), -(b1i - e2r));
            const size_t tot = (size_t)2 * nmaps * P.nrings * M1;
            delta[SHT_IDX(P.dbg, ((size_t)(2 * (b0 + b)) * P.nrings + ring) * M1 + m, tot, 107)] = dq;
            delta[SHT_IDX(P.dbg, ((size_t)(2 * (b0 + b) + 1) * P.nrings + ring) * M1 + m, tot, 107)] = du;
        }
    }
}

template <int BC>
__global__ void __launch_bounds__(kThreads)
legendre_spin2_fp64_kernel(const __grid_constant__ DevPlan P, const double2 *__restrict__ elm,
                           const double2 *__restrict__ blm, double2 *__restrict__ delta, int nmaps)
{
    __shared__ double sA[kChunk];
    __shared__ double2 sx[kChunk][BC][4];
    legendre_spin2_item<BC>(P, elm, blm, delta, nmaps, blockIdx.y, blockIdx.x, blockIdx.z * BC, sA, sx);
}

// Orders mlist[blockIdx.y] only, written through row_off (an m-partition of
// Algorithm 3); the arithmetic of every (m, ring pair) is the full launch's.
template <int BC>
__global__ void __launch_bounds__(kThreads)
legendre_mpart_fp64_kernel(const __grid_constant__ DevPlan P, const double2 *__restrict__ alm,
                           double2 *__restrict__ delta, int nmaps, const int *__restrict__ mlist, int nm,
                           const long long *__restrict__ row_off)
{
    __shared__ double sA[kChunk];
    __shared__ double2 sa[kChunk][BC];
    OutMap om;
    om.row_off = row_off;
    om.bstride = nm;
    om.col = blockIdx.y;
    legendre_item<BC>(P, alm, delta, nmaps, mlist[blockIdx.y], blockIdx.x, blockIdx.z * BC, sA, sa, om);
}

__global__ void delta_gather_kernel(const double2 *__restrict__ src, double2 *__restrict__ dst, int nmaps, int nrows,
                                    int M1, const long long *__restrict__ m_off, const int *__restrict__ m_cnt,
                                    const int *__restrict__ m_col)
{
    const long long total = (long long)nmaps * nrows * M1;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(t % M1);
        const long long br = t / M1;  // b nrows + row
        const int row = (int)(br % nrows), b = (int)(br / nrows);
        dst[t] = src[m_off[m] + ((long long)row * nmaps + b) * m_cnt[m] + m_col[m]];
    }
}

// Many requests (one map each) in one persistent launch: CTAs take work
// items (request, m, ring block) from a list sorted by decreasing cost
// through an atomic counter, so uneven requests balance over the SMs.
__global__ void __launch_bounds__(kThreads)
legendre_multi_fp64_kernel(const DevPlan *__restrict__ plans, const int4 *__restrict__ items, int nitems,
                           int *__restrict__ counter, const MultiPtrs ptrs)
{
    __shared__ double sA[kChunk];
    __shared__ double2 sa[kChunk][1];
    __shared__ int s_item;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int4 w = items[it];  // (request, m, ring block, -)
        legendre_item<1>(plans[w.x], static_cast<const double2 *>(ptrs.alm[w.x]),
                         static_cast<double2 *>(ptrs.delta[w.x]), 1, w.y, w.z, 0, sA, sa);
    }
}

template <int BC>
cudaError_t launch_bc(const DevPlan &P, const double2 *alm, double2 *delta, int nmaps,
                      cudaStream_t st)
{
    dim3 grid((P.npairs + kThreads - 1) / kThreads, P.mmax + 1, (nmaps + BC - 1) / BC);
    legendre_fwd_fp64_kernel<BC><<<grid, kThreads, 0, st>>>(P, alm, delta, nmaps);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_legendre_multi_fp64(const DevPlan *plans, const int4 *items, int nitems, int *counter,
                                       const MultiPtrs &ptrs, int nctas, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    legendre_multi_fp64_kernel<<<nctas, kThreads, 0, st>>>(plans, items, nitems, counter, ptrs);
    return cudaGetLastError();
}

cudaError_t launch_legendre_mpart_fp64(const DevPlan &P, const double2 *alm, double2 *delta, int nmaps,
                                       const int *mlist, int nm, const long long *row_off, cudaStream_t st)
{
    if (nmaps <= 0 || nm <= 0) return cudaSuccess;
    const int bc = nmaps >= 8 ? 8 : nmaps >= 4 ? 4 : nmaps >= 2 ? 2 : 1;
    dim3 grid((P.npairs + kThreads - 1) / kThreads, nm, (nmaps + bc - 1) / bc);
    if (bc == 8)
        legendre_mpart_fp64_kernel<8><<<grid, kThreads, 0, st>>>(P, alm, delta, nmaps, mlist, nm, row_off);
    else if (bc == 4)
        legendre_mpart_fp64_kernel<4><<<grid, kThreads, 0, st>>>(P, alm, delta, nmaps, mlist, nm, row_off);
    else if (bc == 2)
        legendre_mpart_fp64_kernel<2><<<grid, kThreads, 0, st>>>(P, alm, delta, nmaps, mlist, nm, row_off);
    else
        legendre_mpart_fp64_kernel<1><<<grid, kThreads, 0, st>>>(P, alm, delta, nmaps, mlist, nm, row_off);
    return cudaGetLastError();
}

cudaError_t launch_legendre_spin2_fp64(const DevPlan &P, const double2 *elm, const double2 *blm, double2 *delta,
                                       int nmaps, cudaStream_t st)
{
    if (nmaps <= 0) return cudaSuccess;
    const int bc = nmaps >= 2 ? 2 : 1;
    dim3 grid((P.npairs + kThreads - 1) / kThreads, P.mmax + 1, (nmaps + bc - 1) / bc);
    if (bc == 2)
        legendre_spin2_fp64_kernel<2><<<grid, kThreads, 0, st>>>(P, elm, blm, delta, nmaps);
    else
        legendre_spin2_fp64_kernel<1><<<grid, kThreads, 0, st>>>(P, elm, blm, delta, nmaps);
    return cudaGetLastError();
}

cudaError_t launch_delta_gather(const double2 *src, double2 *dst, int nmaps, int nrows, int mmax,
                                const long long *m_off, const int *m_cnt, const int *m_col, cudaStream_t st)
{
    const long long total = (long long)nmaps * nrows * (mmax + 1);
    if (total <= 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 16);
    delta_gather_kernel<<<blocks, 256, 0, st>>>(src, dst, nmaps, nrows, mmax + 1, m_off, m_cnt, m_col);
    return cudaGetLastError();
}

cudaError_t launch_legendre_fwd_fp64(const DevPlan &P, const double2 *alm, double2 *delta,
                                     int nmaps, int bc, cudaStream_t st)
{
    if (nmaps <= 0) return cudaSuccess;
    if (bc <= 0) bc = 8;  // default: 8 maps per CTA
    while (bc > 1 && bc > nmaps) bc /= 2;
    if (bc >= 8) return launch_bc<8>(P, alm, delta, nmaps, st);
    if (bc >= 4) return launch_bc<4>(P, alm, delta, nmaps, st);
    if (bc >= 2) return launch_bc<2>(P, alm, delta, nmaps, st);
    return launch_bc<1>(P, alm, delta, nmaps, st);
}

}  // namespace sht
