// Internal declarations shared by the CUDA translation units of libsht.
// Nothing here is part of the C ABI (see include/sht.h).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace sht {

// Exponent tracking of the Legendre recurrence (Algorithm 2 of the paper,
// real-time rescaling).  A value v carried with exponent k stands for
// v * 2^(kScaleUnit * k).  While k < 0 the value is below 2^-256 and its
// contribution to Delta_m is dropped; when |v| exceeds 2^kScaleHi the pair
// (p_l, p_{l-1}) is multiplied by 2^-kScaleUnit and k is incremented.  Powers
// of two are exact, so the rescaling changes no rounding.
constexpr int kScaleUnit = 512;
constexpr int kScaleHi = 256;

// Debug builds (compiled with -DSHT_DEBUG, see build.py): index checks on the
// kernels' tile, stage, shared-memory, tensor-memory and global offsets.  A
// failed check counts in the plan's debug words (dbg[0] = violations, dbg[1]
// = tag of the first, dbg[2] = its index, dbg[3] = its bound) and the index
// is clamped to 0, so the kernel goes on without touching memory outside its
// buffers (no trap).  Release builds compile the checks away.
#ifdef SHT_DEBUG
__device__ __forceinline__ long long sht_dbg_idx(unsigned long long *dbg, long long i, long long n, int tag)
{
    if (i >= 0 && i < n) return i;
    if (dbg && atomicAdd(dbg, 1ull) == 0ull) {
        dbg[1] = (unsigned long long)tag;
        dbg[2] = (unsigned long long)i;
        dbg[3] = (unsigned long long)n;
    }
    return 0;
}
#define SHT_IDX(dbg, i, n, tag) sht_dbg_idx((dbg), (long long)(i), (long long)(n), (tag))
#define SHT_CHECK(dbg, cond, tag) ((cond) ? (void)0 : (void)sht_dbg_idx((dbg), -1, 0, (tag)))
#else
#define SHT_IDX(dbg, i, n, tag) ((void)(n), (i))
#define SHT_CHECK(dbg, cond, tag) ((void)0)
#endif

// Device-side view of a plan, passed by value to every kernel.
struct DevPlan {
    int lmax, mmax, nrings, npairs;
    long long nalm, npix;
    int max_nphi;   // longest ring
    int fft_cap;    // complex elements per shared-memory FFT buffer
    // ring pairs: the Legendre step runs once per pair of mirrored rings
    const double *pair_x;   // [npairs] cos(theta) of the pair's northern ring
    const int2 *pair_ring;  // [npairs] (northern ring, southern ring or -1)
    // lambda_mm (Eq. pmm) for every (m, pair), as (mantissa, exponent k)
    const double *start_v;  // [mmax+1][npairs]
    const int *start_k;     // [mmax+1][npairs]
    // scaled recurrence p_l = A_l x p_{l-1} - p_{l-2}, lambda_l = C_l p_l,
    // packed m-major like the coefficients (entry (l, m) holds A_l, C_l)
    const double *coefA;
    const double *coefC;
    // rings
    const int *nphi;         // [nrings]
    const long long *ofs;    // [nrings] first pixel
    const double *phi0;      // [nrings]
    const int *ps;           // [nrings] phi0 = pi * ps / nphi, or -1 (arbitrary phi0)
    const double *wring;     // [nrings] quadrature weight of each pixel of the ring (0: none)
    // Evanescent skip of the tensor-core forms (nullptr: none): work item
    // (m, ring block rb) starts at degree m + 64 skip_g[m nrb + rb], where the
    // recurrence state of pair r is (warm_p0, warm_p1, warm_k)[m npairs + r]
    // (p_{l-1}, p_l, exponent); every value below that degree, in every ring of
    // the block, rounds to zero in FP32.
    const int *skip_g;
    const double *warm_p0, *warm_p1;
    const int *warm_k;
    // Orders of the tensor-core forms' Delta that can be nonzero (nullptr: all,
    // set with the skip tables): Delta_m of ring r is exactly zero for
    // m >= ring_mlim[r], because every recurrence value of the ring's pair at
    // those orders rounds to zero in FP32.  The Legendre launches leave out the
    // items whose order is past every ring of their block, so those Delta
    // entries are never written, and the FP32 ring kernels read m < ring_mlim[r].
    const int *ring_mlim;
    const int *block_mlim;  // [nrb] the largest ring_mlim of each block of 128 ring pairs
    // Work lists of the persistent tensor-core launches (sched_ctas == 0:
    // round robin): CTA b of sched_ctas runs items sched_items[sched_off[b] ..
    // sched_off[b + 1]), item = m nrb + rb.  The lists replay a work queue
    // served in m order to the CTA with the least work so far, so every CTA
    // gets the same work to within one item (whatever the skip leaves of each)
    // and the ring blocks of one order still run at about the same time,
    // sharing its B operand in L2.
    const int *sched_off;
    const int *sched_items;
    int sched_ctas;
    const long long *twofs;  // [nrings] offset of the ring's table in tw64 / tw32
    const double2 *tw64;     // per distinct nphi = n: e^{i pi q / n}, q in [0, 2n)
    const float2 *tw32;
    // Rings whose FFT length N has a large prime factor run Bluestein's
    // algorithm (two power-of-two FFTs of length Mb >= 2N - 1 around a
    // pointwise product with the FFT of the chirp); the others the direct
    // mixed-radix transform.  Each set is launched over its own ring list.
    int n_smooth, n_blue;
    const int *rings_smooth;   // [n_smooth]
    const int *rings_blue;     // [n_blue]
    const int *blue_mb;        // [nrings] Mb (0 for smooth rings)
    const long long *blue_ofs; // [nrings] offset of the ring's chirp spectrum in bhat64 / bhat32
    const long long *chirp_ofs;  // [nrings] offset of the ring's chirp e^{i pi t^2 / N}, t < N, in chirp32
    const float2 *chirp32;
    const double2 *bhat64;     // per distinct Bluestein N: FFT_Mb(e^{-i pi t^2 / N}, wrapped) / Mb
    const float2 *bhat32;
    const double2 *w2_64;      // e^{2 pi i q / kBlueMaxMb}, q < kBlueMaxMb
    const float2 *w2_32;
    int blue_cap;              // largest Mb (0 if none)
    // FP32 ring step with the FFT in registers (ring_reg.cu): rf_len[r] = L for
    // a direct transform of length L = n / 2 (a power of two, 256..4096), -L for
    // Bluestein's algorithm with a power-of-two length L (n / 2 <= 2048), 0 for a
    // ring left to the shared-memory kernel (odd n, or no such L).  Bluestein
    // rings: chirp e^{i pi t^2 / N}, t < N = n / 2, at rf_ch32 + rf_ch_ofs[r] and
    // FFT_L(e^{-i pi t^2 / N}, wrapped) / L at rf_bh32 + rf_bh_ofs[r].
    const int *rf_len;
    const long long *rf_ch_ofs, *rf_bh_ofs;
    const float2 *rf_ch32, *rf_bh32;
    const int *rf_rings;       // [rf_n] the rings with rf_len != 0, by decreasing cost
    int rf_n;
    // the rings with rf_len == 0, split as rings_smooth / rings_blue are
    const int *rf_rest_smooth, *rf_rest_blue;
    int rf_n_rest_smooth, rf_n_rest_blue;
    // FP64 ring step over a ring partition (sht_ring_synth_part): Delta row of
    // ring r is ring_row[r] of delta_rows per map (ring_row == nullptr: row r of nrings)
    const int *ring_row;
    int delta_rows;
    unsigned long long *dbg;  // debug words of the index checks (nullptr unless built with SHT_DEBUG)
};
// Largest order of ring r whose FP32 Delta can be nonzero (DevPlan::ring_mlim).
__device__ __forceinline__ int ring_mtop(const DevPlan &P, int r)
{
    return P.ring_mlim ? min(P.mmax, P.ring_mlim[r] - 1) : P.mmax;
}
constexpr int kBlueMinPrime = 29;  // a prime factor at least this large selects Bluestein
constexpr int kBlueMaxMb = 4096;   // largest Bluestein FFT length (shared-memory bound)

// Per-request device pointers of a multi-request call (kernel parameter).
constexpr int kMaxReq = 256;
struct MultiPtrs {
    const void *alm[kMaxReq];
    void *map[kMaxReq];
    void *delta[kMaxReq];
};

// Legendre step, FP64 (recurrence and contraction in FP64).
//   delta[b][ring][m] (complex) = Delta_m(theta_ring) for maps b in [0, nmaps);
//   bc = maps per CTA (1, 2, 4, 8; 0 = 8), a tile shape only: results do not depend on it.
cudaError_t launch_legendre_fwd_fp64(const DevPlan &P, const double2 *alm, double2 *delta,
                                     int nmaps, int bc, cudaStream_t st);

// Legendre step in FP64 for the orders mlist[0..nm) only (an m-partition):
// Delta_{mlist[i]} of ring r and map b goes to delta[row_off[r] + b nm + i]
// (complex128), row_off[r] laying out the rings for an all-to-all exchange.
cudaError_t launch_legendre_mpart_fp64(const DevPlan &P, const double2 *alm, double2 *delta, int nmaps,
                                       const int *mlist, int nm, const long long *row_off, cudaStream_t st);
// Spin-2 Legendre step (polarisation), FP64: E, B [map][nalm] complex128 ->
// Delta of Q and U, delta[((2 b + q) nrings + ring) (mmax + 1) + m], q = 0 (Q), 1 (U);
// the ring step then runs on 2 nmaps "maps" and writes [map][Q, U][npix].
cudaError_t launch_legendre_spin2_fp64(const DevPlan &P, const double2 *elm, const double2 *blm, double2 *delta,
                                       int nmaps, cudaStream_t st);
// Gather of the exchanged blocks into the ring step's layout: for order m,
// rows of the partition's rings, maps b:
//   dst[(b nrows + row) (mmax + 1) + m] = src[m_off[m] + (row nmaps + b) m_cnt[m] + m_col[m]].
cudaError_t launch_delta_gather(const double2 *src, double2 *dst, int nmaps, int nrows, int mmax,
                                const long long *m_off, const int *m_cnt, const int *m_col, cudaStream_t st);

// Legendre step of many one-map requests in one persistent launch over the
// work list items[] = (request, m, ring block, -); counter must be 0 at launch.
cudaError_t launch_legendre_multi_fp64(const DevPlan *plans, const int4 *items, int nitems, int *counter,
                                       const MultiPtrs &ptrs, int nctas, cudaStream_t st);
// Ring step of many requests: one launch over items (request, ring) of rings
// with a direct transform, one over rings run with Bluestein's algorithm.
cudaError_t launch_ring_synth_multi_fp64(const DevPlan *plans, const int2 *smooth_items, int n_smooth,
                                         int smooth_cap, const int2 *blue_items, int n_blue, int blue_cap,
                                         const MultiPtrs &ptrs, cudaStream_t st);

// Ring step: phase shift, fold of m onto the ring's bins, real inverse DFT of
// each ring; delta is [map][ring][m].
// FP32 ring step reading the tensor-core layout [ring][m][map] directly,
// g_smooth / g_blue maps (1, 2 or 4) per CTA for the two ring lists, nt
// (256 or 512) threads per CTA; the shared memory per CTA is
// ring_mf_smem_bytes(cap, G).
cudaError_t launch_ring_synth_mf(const DevPlan &P, const float2 *delta_rm, float *map, int nmaps, int g_smooth,
                                 int g_blue, int nt, cudaStream_t st);
size_t ring_mf_smem_bytes(int cap, int G);
// group = maps per CTA (0 = 8), a tile shape only.
cudaError_t launch_ring_synth_fp64(const DevPlan &P, const double2 *delta, double *map, int nmaps, int group,
                                   cudaStream_t st);

// Ring step of the transpose: q[b][ring][m] = sum_j y_j e^{-i m phi_j}.
cudaError_t launch_ring_analysis_fp64(const DevPlan &P, const double *map, double2 *q, int nmaps,
                                      const double *wring, cudaStream_t st);
// The same ring step of the transpose in FP32 (the tensor-core forms' maps);
// group = maps per CTA (a tile shape: results do not depend on it).
cudaError_t launch_ring_analysis_fp32(const DevPlan &P, const float *map, float2 *q, int nmaps,
                                      const double *wring, int group, cudaStream_t st);
// Legendre step of the transpose, FP64:
//   g[b][idx(l, m)] = c_m sum_r lambda_lm(x_r) q[b][r][m],  c_0 = 1, c_m = cfac for m > 0
//   (cfac = 2: the real-linear transpose of alm2map; cfac = 1: the analysis sum).
cudaError_t launch_legendre_adj_fp64(const DevPlan &P, const double2 *q, double2 *g, int nmaps, double cfac,
                                     cudaStream_t st);
// Shared memory the FP64 adjoint Legendre kernel needs (0 if the plan has too many ring pairs).
size_t legendre_adj_smem_bytes(const DevPlan &P, int bc);

// Tensor-core Legendre step (precision forms).  Per launch group of at most
// kTcMaxMaps maps, the B operand (C_l a_lm split into TF32 / BF16 pieces) is
// laid out per (m, parity) segment of padded length K in bbuf; seg_* hold the
// segment offsets ([mmax+1][2]) for the TF32 (K chunk 8) and BF16 (K chunk 16)
// layouts, kall_* the total padded K.  status: device word set to SHT_ETIMEOUT
// when a bounded device-side wait gives up.
constexpr int kTcMaxMaps = 64;
struct TcWork {
    const int *seg_tf32 = nullptr;
    const int *seg_bf16 = nullptr;
    int withhold = -1;  // test hook: stage whose copies CTA 0 of the next launch skips (-1: none)
    long long kall_tf32 = 0, kall_bf16 = 0;
    void *bbuf = nullptr;
    int *status = nullptr;
};
__host__ __device__ inline int tc_ncols(int nmaps) { return ((2 * nmaps + 31) / 32) * 32; }

// Per-request operands of a many-request tensor-core launch (one map each).
struct MultiTcPtrs {
    const void *alm[kMaxReq];   // the request's coefficients, complex128
    const void *bbuf[kMaxReq];  // B operand image of the request's plan
    const int *seg[kMaxReq];    // its (m, parity) segment table for the form
    void *delta[kMaxReq];       // its Delta, complex64 [ring][m]
    void *map[kMaxReq];         // its map, float32
    // work lists: the items are stored CTA-major, CTA b of ctas running items
    // [cta_off[b], cta_off[b + 1]) (ctas == 0: round robin)
    const int *cta_off;
    int ctas;
};
size_t tc_bbuf_bytes(const TcWork &W, int prec);
cudaError_t launch_tc_prep(const DevPlan &P, const TcWork &W, int prec, const double2 *alm, int nmaps,
                           cudaStream_t st);
// Operand prep of many one-map requests in one launch over items (request, m).
cudaError_t launch_tc_prep_multi(const DevPlan *plans_dev, const int2 *items, int nitems, const MultiTcPtrs &mp,
                                 int prec, cudaStream_t st);
// delta: [ring][m][map] for the launch's nmaps maps (a row's maps contiguous,
// so every store fills whole sectors).  acache: the plan-time Lambda operand
// of form prec (launch_lambda_build), or nullptr to run the FP64 recurrence in
// the launch.
cudaError_t launch_tc_main(const DevPlan &P, const TcWork &W, int prec, const void *acache, float2 *delta,
                           int nmaps, cudaStream_t st);
// Many requests (one map each) in one persistent launch: items (request, m,
// ring block) sorted by decreasing cost; plans_dev[request] are the requests'
// plans (with their skip tables), P any one of them (launch shape only).
cudaError_t launch_tc_main_multi(const DevPlan &P, const DevPlan *plans_dev, const int4 *items, int nitems,
                                 const MultiTcPtrs &mp, int prec, int *status, cudaStream_t st);
// FP32 ring step of many requests (one map each, Delta [ring][m]): items
// (request, ring) of the smooth and Bluestein lists; caps are the largest
// buffers over the requests.
cudaError_t launch_ring_synth_mf_multi(const DevPlan *plans_dev, const int2 *smooth_items, int n_smooth,
                                       int smooth_cap, const int2 *blue_items, int n_blue, int blue_cap,
                                       const MultiTcPtrs &mp, int nt, cudaStream_t st);
size_t tc_lambda_bytes(const DevPlan &P, const TcWork &W, int prec);
// Fill the evanescent-skip tables (skip_g: [mmax+1][nrb]; warm_*: [mmax+1][npairs])
// and raise pair_lim[pair] (zeroed by the caller) to 1 + the largest order with
// a recurrence value of the pair representable in FP32.
cudaError_t launch_warm_start(const DevPlan &P, int *skip_g, double *warm_p0, double *warm_p1, int *warm_k,
                              int *pair_lim, cudaStream_t st);
cudaError_t launch_lambda_build(const DevPlan &P, const TcWork &W, int prec, void *out, cudaStream_t st);
// Legendre step of the transpose (map2alm_adjoint), BF16 forms, from the
// plan-time Lambda operand acache of the same form: g[map][alm] = c_m C_l
// sum_pairs p_l(x) (q_N + (-1)^{l-m} q_S)(m), c_0 = 1, c_m = cfac, Im g_l0 = 0.  q: FP32 ring
// analysis [map][ring][m] of nmaps <= 32 maps; bimg: workspace of
// adj_tc_bimg_bytes(P, prec, nmaps) bytes; items: (m, block j of 128 degrees
// of each parity) for every m and j < ceil(ceil((lmax - m + 1) / 32) / 8).
// Two launches (operand image, contraction).
size_t adj_tc_bimg_bytes(const DevPlan &P, int prec, int nmaps);
cudaError_t launch_adj_tc(const DevPlan &P, const TcWork &W, int prec, const void *acache, const float2 *q,
                          void *bimg, const int2 *items, int nitems, double2 *g, int nmaps, double cfac,
                          cudaStream_t st);

// FP32 ring step of the tensor-core forms with the FFT in registers, over the
// plan's rf_rings (Delta [ring][m][map] for nmaps maps); status gets
// SHT_ETIMEOUT if a bounded wait for a Delta copy runs out.  The rings outside
// rf_rings are left to launch_ring_synth_mf with the rf_rest lists.
cudaError_t launch_ring_reg(const DevPlan &P, const float2 *delta_rm, float *map, int nmaps, int *status,
                            cudaStream_t st);
// The same over (request, ring) items of one-map requests (items ordered by
// decreasing cost); max_mmax is the largest mmax over the requests, P any of them.
cudaError_t launch_ring_reg_multi(const DevPlan &P, const DevPlan *plans_dev, const int2 *items, int nitems,
                                  int max_mmax, const MultiTcPtrs &mp, int *status, cudaStream_t st);
// Dynamic shared memory of that kernel for a plan's mmax.
size_t ring_reg_smem_bytes(int mmax);

// Kernels one ring-step launch issues (one per non-empty ring list).
inline int ring_launches(const DevPlan &P) { return (P.n_smooth > 0) + (P.n_blue > 0); }

// Shared-memory bytes the ring kernels need for this plan.
inline size_t ring_smem_bytes_for_cap(int cap, bool fp64)
{
    return (size_t)3 * cap * (fp64 ? 16 : 8);  // two FFT buffers + twiddle table
}

}  // namespace sht
