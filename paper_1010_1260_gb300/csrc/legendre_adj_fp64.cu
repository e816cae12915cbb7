// Legendre step of the transpose (map2alm_adjoint) in FP64:
//   g_lm = c_m sum_r lambda_lm(x_r) q_m(r),  c_0 = 1, c_m = 2 for m > 0 (c_m = 1
//   for the quadrature-weighted analysis sum, whose q carries the weights),
// the real-linear transpose of Eq. DeltaDef (the paper's map2alm, Eq. map2almDef,
// without quadrature weights).  With the ring pairs of the forward step and
// lambda_lm(-x) = (-1)^(l-m) lambda_lm(x):
//   g_lm = c_m C_l sum_pairs p_l(x) (q_N + (-1)^(l-m) q_S).
//
// Mapping (GB300): one CTA per (m, group of BC maps).  The sum over ring pairs
// is a reduction, so the CTA works in tiles instead of one pair per thread:
// for each chunk of 32 degrees l and each block of 128 ring pairs,
//   phase 1: thread t advances pair t's recurrence over the 32 l (FP64,
//            exponent-tracked as in the forward kernel) and writes p_l into a
//            shared 128 x 32 tile (zero while the pair is still rescaled);
//   phase 2: thread (l, map, pair-slice) contracts its tile column with the
//            pairs' (q_N + q_S, q_N - q_S) -- no cross-thread reduction.
// The recurrence state of every pair lives in shared memory between chunks.
// FP64 work is exactly the algorithmic 2 ops per (l, pair) for the recurrence
// plus 2 per (l, pair, map) for the contraction.
#include "sht_internal.cuh"

namespace sht {
namespace {

constexpr int kThreads = 128;
constexpr int kCL = 32;        // degrees per chunk (even)
constexpr int kPB = kThreads;  // ring pairs per tile
constexpr int kLamStride = kCL + 1;

__device__ __forceinline__ bool above_hi(double v)
{
    const int e = (__double2hiint(v) >> 20) & 0x7ff;
    return e > 1023 + kScaleHi;
}

struct QPair {
    double2 e, o;  // q_N + q_S and q_N - q_S
};

template <int BC>
__global__ void __launch_bounds__(kThreads)
legendre_adj_fp64_kernel(const DevPlan P, const double2 *__restrict__ q, double2 *__restrict__ g,
                         int nmaps, double cfac)
{
    constexpr int PS = 4 / BC;  // pair slices in phase 2
    const int m = blockIdx.x;
    const int b0 = blockIdx.y * BC;
    const int L = P.lmax;
    const int M1 = P.mmax + 1;
    const int R = P.npairs;
    const int tid = threadIdx.x;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *st_p0 = reinterpret_cast<double *>(smem_raw);
    double *st_p1 = st_p0 + R;
    double *lam = st_p1 + R;                                      // [kPB][kLamStride]
    QPair *qs = reinterpret_cast<QPair *>(lam + kPB * kLamStride);  // [kPB][BC]
    double2 *red = reinterpret_cast<double2 *>(qs + kPB * BC);      // [kThreads]
    double *sA = reinterpret_cast<double *>(red + kThreads);        // [kCL]
    int *st_k = reinterpret_cast<int *>(sA + kCL);                  // [R]

    for (int p = tid; p < R; p += kThreads) {
        st_p0[p] = 0.0;
        st_p1[p] = P.start_v[(size_t)m * R + p];
        st_k[p] = P.start_k[(size_t)m * R + p];
    }

    const int lj = tid % kCL;         // phase-2 degree slot
    const int bsel = (tid / kCL) % BC;  // phase-2 map
    const int ph = tid / (kCL * BC);    // phase-2 pair slice
    const long long mofs = (long long)m * (2 * L + 3 - m) / 2;
    const double cm = (m == 0) ? 1.0 : cfac;

    for (int l0 = m; l0 <= L; l0 += kCL) {
        const int cnt = min(kCL, L + 1 - l0);
        __syncthreads();
        for (int i = tid; i < cnt; i += kThreads) {
            const int l = l0 + i;
            sA[i] = (l + 1 <= L) ? P.coefA[mofs + (l + 1 - m)] : 0.0;
        }
        double2 acc = make_double2(0.0, 0.0);
        for (int pb = 0; pb < R; pb += kPB) {
            __syncthreads();
            // phase 1: recurrence of pair pb + tid over this chunk
            const int pair = pb + tid;
            double *row = lam + tid * kLamStride;
            if (pair < R) {
                const double x = P.pair_x[pair];
                double p0 = st_p0[pair], p1 = st_p1[pair];
                int k = st_k[pair];
                for (int j = 0; j < cnt; ++j) {
                    row[j] = (k == 0) ? p1 : 0.0;
                    const double t = fma(sA[j] * x, p1, -p0);
                    p0 = p1;
                    p1 = t;
                    if (k < 0 && above_hi(p1)) {
                        p1 *= 0x1p-512;
                        p0 *= 0x1p-512;
                        k += 1;
                    }
                }
                st_p0[pair] = p0;
                st_p1[pair] = p1;
                st_k[pair] = k;
                const int2 rr = P.pair_ring[pair];
#pragma unroll
                for (int b = 0; b < BC; ++b) {
                    double2 qn = make_double2(0.0, 0.0), qsv = make_double2(0.0, 0.0);
                    if (b0 + b < nmaps) {
                        const double2 *qb = q + (size_t)(b0 + b) * P.nrings * M1;
                        qn = qb[(size_t)rr.x * M1 + m];
                        if (rr.y >= 0) qsv = qb[(size_t)rr.y * M1 + m];
                    }
                    QPair v;
                    v.e = make_double2(qn.x + qsv.x, qn.y + qsv.y);
                    v.o = make_double2(qn.x - qsv.x, qn.y - qsv.y);
                    qs[tid * BC + b] = v;
                }
            } else {
                for (int j = 0; j < cnt; ++j) row[j] = 0.0;
#pragma unroll
                for (int b = 0; b < BC; ++b) {
                    QPair v;
                    v.e = make_double2(0.0, 0.0);
                    v.o = v.e;
                    qs[tid * BC + b] = v;
                }
            }
            __syncthreads();
            // phase 2: column lj of the tile against this slice of pairs
            if (lj < cnt) {
                const bool odd = lj & 1;  // (l - m) parity: chunks start at even l - m
                const int plo = ph * (kPB / PS), phi = plo + kPB / PS;
#pragma unroll 4
                for (int p = plo; p < phi; ++p) {
                    const double lv = lam[p * kLamStride + lj];
                    const QPair v = qs[p * BC + bsel];
                    const double2 qq = odd ? v.o : v.e;
                    acc.x = fma(lv, qq.x, acc.x);
                    acc.y = fma(lv, qq.y, acc.y);
                }
            }
        }
        // combine the pair slices and write g for this chunk
        __syncthreads();
        red[tid] = acc;
        __syncthreads();
        if (ph == 0 && lj < cnt && b0 + bsel < nmaps) {
            double2 s = acc;
            for (int h = 1; h < PS; ++h) {
                const double2 o = red[tid + h * kCL * BC];
                s.x += o.x;
                s.y += o.y;
            }
            const long long idx = mofs + (l0 - m) + lj;
            const double c = cm * P.coefC[idx];
            g[(size_t)(b0 + bsel) * P.nalm + idx] = make_double2(c * s.x, (m == 0) ? 0.0 : c * s.y);
        }
    }
}

template <int BC>
size_t smem_bytes(int R)
{
    return (size_t)R * (8 + 8 + 4) + (size_t)kPB * kLamStride * 8 + (size_t)kPB * BC * sizeof(QPair) +
           (size_t)kThreads * 16 + (size_t)kCL * 8 + 16;
}

template <int BC>
cudaError_t launch_bc(const DevPlan &P, const double2 *q, double2 *g, int nmaps, double cfac, cudaStream_t st)
{
    const size_t smem = smem_bytes<BC>(P.npairs);
    auto kern = legendre_adj_fp64_kernel<BC>;
    if (smem > 40 * 1024) {  // dynamic + static above the 48 KB default needs the opt-in
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(P.mmax + 1, (nmaps + BC - 1) / BC);
    kern<<<grid, kThreads, smem, st>>>(P, q, g, nmaps, cfac);
    return cudaGetLastError();
}

int pick_bc(int nmaps) { return nmaps >= 4 ? 4 : (nmaps >= 2 ? 2 : 1); }

}  // namespace

size_t legendre_adj_smem_bytes(const DevPlan &P, int bc)
{
    const size_t s = bc >= 4 ? smem_bytes<4>(P.npairs) : (bc == 2 ? smem_bytes<2>(P.npairs) : smem_bytes<1>(P.npairs));
    return s <= (size_t)(227 * 1024 - 1024) ? s : 0;
}

cudaError_t launch_legendre_adj_fp64(const DevPlan &P, const double2 *q, double2 *g, int nmaps, double cfac,
                                     cudaStream_t st)
{
    if (nmaps <= 0) return cudaSuccess;
    const int bc = pick_bc(nmaps);
    if (bc == 4) return launch_bc<4>(P, q, g, nmaps, cfac, st);
    if (bc == 2) return launch_bc<2>(P, q, g, nmaps, cfac, st);
    return launch_bc<1>(P, q, g, nmaps, cfac, st);
}

}  // namespace sht
