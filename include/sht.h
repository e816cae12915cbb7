/*
 * sht.h -- C ABI of libsht: the inverse spherical harmonic transform
 * (alm2map) and its real-linear transpose on one NVIDIA GB300 (sm_103a).
 *
 * Method: Hupca, Falcou, Grigori, Stompor, "Spherical harmonic transform with
 * GPUs" (INRIA RR-7409).  alm2map evaluates Eq. alm2mapDef,
 *     s(theta, phi) = sum_{l <= lmax} sum_{|m| <= l} a_lm Y_lm(theta, phi),
 * on an iso-latitude ring grid in the two steps of Algorithm 1: the Legendre
 * step forms Delta_m(theta_r) of Eq. DeltaDef with the recurrence of
 * Eq. assLegRec (starting values Eq. pmm / Eq. pm1m, rescaled against
 * underflow as in Algorithm 2), and the ring step sums Eq. Delta2map with one
 * FFT per ring (sec. 2.2.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Coefficients (alm): complex128, interleaved (re, im), m-major packed:
 *     idx(l, m) = m (2 lmax + 3 - m) / 2 + (l - m),  0 <= m <= mmax, m <= l <= lmax,
 *   nalm = (mmax + 1)(2 lmax + 2 - mmax) / 2 entries per map; map b of a batch
 *   starts at entry b * nalm.  Y_lm = lambda_lm(cos theta) e^{i m phi} with
 *   orthonormal lambda_lm including the Condon-Shortley sign (-1)^m.  The map
 *   is real (sec. 2.1), so Im(a_l0) is ignored and a_{l,-m} = (-1)^m conj(a_lm)
 *   is implied.
 * Maps: real, RING order (rings north to south, pixels by increasing phi
 *   within a ring); npix pixels per map, map b starts at pixel b * npix.
 *   float64 for SHT_FP64, float32 for the tensor-core forms.
 * Pointers named *_dev are device pointers on the plan's device; the caller
 *   owns them and the library never frees them.  The library owns the plan,
 *   its tables and its workspace (allocated at plan time or grown on first use
 *   of a larger batch).
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Launches are asynchronous; calls on one plan must be ordered on
 *   one stream (they share the plan's workspace).
 * Errors: every int-returning call returns SHT_OK (0) or a negative code; the
 *   calling thread's message is available from sht_last_error().  Bad
 *   arguments are rejected before anything is launched.
 */
#ifndef SHT_H
#define SHT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SHT_OK 0
#define SHT_EINVAL (-1)       /* bad argument (null pointer, size, kind) */
#define SHT_ENOMEM (-2)       /* host or device allocation failed */
#define SHT_ECUDA (-3)        /* a CUDA call failed */
#define SHT_EUNSUPPORTED (-4) /* valid but not supported (e.g. ring too long) */
#define SHT_ETIMEOUT (-5)     /* a bounded device-side wait gave up */

typedef struct sht_plan_s *sht_plan_t;

typedef enum {
    SHT_GRID_GL = 0,      /* Gauss-Legendre rings, nphi_gl equispaced pixels, phi0 = 0 */
    SHT_GRID_HEALPIX = 1, /* HEALPix RING scheme (Gorski et al. 2005), 4 nside - 1 rings */
    SHT_GRID_RINGS = 2    /* caller-given rings: theta, nphi, phi0 (copied at plan time) */
} sht_grid_kind;

typedef struct {
    int kind;            /* sht_grid_kind */
    int nside;           /* HEALPIX: nside >= 1 */
    int nrings;          /* GL, RINGS: number of rings >= 1 */
    int nphi_gl;         /* GL: pixels per ring >= 1 */
    const double *theta; /* RINGS: host array [nrings], colatitudes in [0, pi] */
    const int *nphi;     /* RINGS: host array [nrings], pixels per ring >= 1 */
    const double *phi0;  /* RINGS: host array [nrings], azimuth of pixel 0 */
} sht_grid;

typedef enum {
    SHT_FP64 = 0,      /* FP64 recurrence, FP64 contraction, FP64 ring FFT; float64 map */
    SHT_FP32_TC = 1,   /* FP64 recurrence, 3xTF32 tensor-core contraction, FP32 ring FFT; float32 map */
    SHT_BF16X3_TC = 2, /* FP64 recurrence, split-BF16 (hi/lo, 3 products) tensor-core contraction,
                          FP32 ring FFT; float32 map.  Does NOT meet a 1e-6 relative-L2 error:
                          two 8-bit pieces carry about 16 significant bits (about 4.9e-6 per
                          map at lmax 2048); use SHT_BF16X6_TC for 1e-6 */
    SHT_BF16X6_TC = 3  /* as SHT_BF16X3_TC with three BF16 pieces and 6 products (hi*hi, hi*mid,
                          mid*hi, hi*lo, mid*mid, lo*hi) */
} sht_prec;

/* Build a plan for grid g and band limits 0 <= mmax <= lmax on the current
 * CUDA device: ring geometry, the recurrence coefficients of Eq. betaDef in
 * the scaled form used by the kernels, the starting values lambda_mm of
 * Eq. pmm with their binary exponents, and the ring-FFT twiddle tables.
 * Limits: lmax <= 8192; every ring's nphi <= 8192.  On success *out holds the
 * plan (free with sht_plan_destroy).  Errors: SHT_EINVAL, SHT_EUNSUPPORTED,
 * SHT_ENOMEM, SHT_ECUDA. */
int sht_plan(const sht_grid *g, int lmax, int mmax, sht_plan_t *out);

/* Free a plan and its device memory (synchronises the plan's device).  NULL is a no-op. */
int sht_plan_destroy(sht_plan_t plan);

/* Sizes: coefficients per map, pixels per map, rings; 0 for a NULL plan. */
size_t sht_nalm(sht_plan_t plan);
size_t sht_npix(sht_plan_t plan);
int sht_nrings(sht_plan_t plan);
int sht_lmax(sht_plan_t plan);
int sht_mmax(sht_plan_t plan);

/* alm2map of one map (Eq. alm2mapDef via Eq. DeltaDef and Eq. Delta2map).
 * alm_dev: nalm complex128 (device); map_dev: npix reals (device), fully
 * overwritten.  prec: sht_prec (selects the map's float type).  The
 * tensor-core forms process batches in groups of up to 64 maps. */
int sht_alm2map(sht_plan_t plan, const void *alm_dev, void *map_dev, int prec, void *stream);

/* Real-linear transpose of alm2map (Eq. map2almDef without quadrature weights):
 *   g_lm = c_m sum_p y_p lambda_lm(theta_p) e^{-i m phi_p},  c_0 = 1, c_m = 2 (m > 0),
 *   Im g_l0 = 0, so that <alm2map(a), y> = sum Re(a) Re(g) + Im(a) Im(g).
 * map_dev: npix reals (float64; float32 for the tensor-core forms); alm_dev:
 * nalm complex128, fully overwritten.
 * prec SHT_FP64: FP64 ring analysis and Legendre accumulation.
 * prec SHT_BF16X6_TC / SHT_BF16X3_TC: FP32 ring analysis, then the Legendre
 * step on the tensor cores as per-m GEMMs over the ring pairs, reading the
 * plan-time Lambda operand of that form transposed; it must have been built
 * (sht_lambda_cache), else SHT_EUNSUPPORTED.  Accuracy as the forward of the
 * form (relative L2 per map about 5e-7 for BF16X6).  The first call
 * allocates the plan's transpose workspace (FP32 ring analysis and operand
 * image of 32 maps: about 5 GB at lmax 2048 on a 4095-ring grid).
 * prec SHT_FP32_TC: SHT_EUNSUPPORTED (its operand would need TF32 operands
 * read MN-major; not built). */
int sht_map2alm_adjoint(sht_plan_t plan, const void *map_dev, void *alm_dev, int prec, void *stream);

/* Quadrature-weighted analysis, map2alm (Eq. map2almDef with the integral's
 * measure and the conjugate harmonic; the paper leaves this direction to
 * future work, sec. 1):
 *   a_lm = sum_p w_p y_p lambda_lm(theta_p) e^{-i m phi_p},  m >= 0,
 * with w_p the plan's pixel weight of p's ring: Gauss-Legendre weight x 2 pi /
 * nphi on a GL grid (exact for band-limited maps when nrings >= lmax + 1 and
 * nphi >= 2 lmax + 1), 4 pi / npix on HEALPix (equal-area pixels; approximate),
 * none on a RINGS grid until sht_set_ring_weights.  niter >= 0 Jacobi
 * refinements a += map2alm(y - alm2map(a)) follow (the usual HEALPix
 * iteration); they allocate two temporary buffers (nbatch maps, nbatch
 * coefficient sets) and synchronise `stream` at the end; they are built for
 * SHT_FP64 only.  prec SHT_BF16X6_TC / SHT_BF16X3_TC (niter = 0): the
 * tensor-core transpose of sht_map2alm_adjoint with the ring weights and
 * c_m = 1 (float32 maps; needs the plan-time Lambda operand of that form).
 * map_dev: nbatch x npix float64 (float32 for the tensor-core forms);
 * alm_dev: nbatch x nalm complex128, fully overwritten.  Errors: SHT_EINVAL,
 * SHT_EUNSUPPORTED (no weights, SHT_FP32_TC, niter > 0 in a tensor-core form,
 * no Lambda operand), SHT_ENOMEM, SHT_ECUDA. */
int sht_map2alm(sht_plan_t plan, const void *map_dev, void *alm_dev, int prec, int niter, void *stream);
int sht_map2alm_batch(sht_plan_t plan, int nbatch, const void *map_dev, void *alm_dev, int prec, int niter,
                      void *stream);

/* Pixel quadrature weight of every ring (host array of nrings doubles, each
 * finite and >= 0): set (synchronises the plan's device) or read. */
int sht_set_ring_weights(sht_plan_t plan, const double *w);
int sht_ring_weights(sht_plan_t plan, double *w);

/* Batched forms of sht_alm2map and sht_map2alm_adjoint (Eq. alm2mapDef and its
 * transpose, map by map): nbatch >= 0 maps stored back to back, alm_dev
 * nbatch x nalm complex128 and map_dev nbatch x npix of the form's map type
 * (float64 for SHT_FP64, float32 otherwise); the caller owns both buffers.
 * nbatch == 0 is a no-op.  Errors as for the single-map calls. */
int sht_alm2map_batch(sht_plan_t plan, int nbatch, const void *alm_dev, void *map_dev,
                      int prec, void *stream);
int sht_map2alm_adjoint_batch(sht_plan_t plan, int nbatch, const void *map_dev, void *alm_dev,
                              int prec, void *stream);

/* Plan-time Lambda operand for one tensor-core form (SHT_FP32_TC,
 * SHT_BF16X3_TC, SHT_BF16X6_TC).  The paper evaluates the recurrence of
 * Eq. assLegRec on the fly inside alm2map (sec. 2.2.2, and the trade of
 * computation against memory traffic in sec. 5); this caches its result
 * instead: every lambda_lm(x_r) of the plan, rounded and split into the
 * form's tensor-core pieces exactly as the recurrence launch makes them, is
 * written once to device memory in the kernel's tile layout.  Later
 * sht_alm2map / sht_alm2map_batch calls of that form on this plan stream the
 * tiles instead of running the recurrence; their results are bit-identical.
 * Size: sht_lambda_cache_bytes(plan, prec) bytes of device memory, about
 * npairs x N_lm x (8, 4, 6) bytes for (FP32_TC, BF16X3_TC, BF16X6_TC): 17-35 GB
 * at lmax 2048 on a 4095-ring grid.
 * enable != 0 builds it (a no-op if present): allocates, launches the build on
 * `stream` and synchronises that stream before returning.  enable == 0 frees
 * it (synchronises the device first).  The plan owns the memory; sht_plan_destroy
 * frees it.  Errors: SHT_EINVAL (no plan, prec not a tensor-core form),
 * SHT_ENOMEM (allocation failed; the plan is unchanged), SHT_ECUDA. */
int sht_lambda_cache(sht_plan_t plan, int prec, int enable, void *stream);

/* Bytes the Lambda operand of form prec needs on this plan; 0 for a NULL plan
 * or a form without one. */
long long sht_lambda_cache_bytes(sht_plan_t plan, int prec);

/* The work lists the persistent tensor-core launches run, computed on the
 * host (no device access): items 0 .. nitems-1, taken in that order, go one
 * by one to the list with the least total cost so far (ties: the lowest list
 * index) -- the replay of a work queue served in item order.  List b is
 * items[off[b] .. off[b + 1] - 1], in item order; off has nlists + 1 entries,
 * items nitems.  Every list's total stays within the largest single cost of
 * the mean.  The library orders a plan's (m, ring block) items by m and a
 * many-request launch's by decreasing cost, with the cost of an item the
 * degrees its recurrence runs after the evanescent skip plus a fixed share for
 * its setup.  Returns SHT_EINVAL for nitems < 0, nlists < 1, a NULL array or
 * a negative cost. */
int sht_work_lists(int nitems, const long long *cost, int nlists, int *off, int *items);

/* Test hook: enable = 0 makes the plan's later tensor-core launches take their
 * work items round robin (CTA b runs items b, b + G, ...) instead of the
 * lists above, enable = 1 restores the lists.  The maps are the same either
 * way (each item's arithmetic does not depend on its CTA); only the balance
 * differs.  SHT_EINVAL for a NULL plan. */
int sht_debug_work_lists(sht_plan_t plan, int enable);

/* Index checks of a debug build (the library compiled with -DSHT_DEBUG,
 * `build(debug=True)`; no counterpart in the paper): the kernels check their
 * tile, stage, tensor-memory, shared-memory and global offsets, count a
 * violation in the plan's device words and clamp the offending index to 0
 * instead of touching memory outside a buffer.  out (host, 5 entries):
 * out[0] = 1 if the library was built with the checks (0: release build,
 * the other entries 0), out[1] = violations since the last report, out[2] =
 * tag of the first (the check's site), out[3] = its index, out[4] = its
 * bound.  Synchronises the device and resets the count.  SHT_EINVAL for a
 * NULL plan or array. */
int sht_debug_report(sht_plan_t plan, unsigned long long *out);

/* Test hook: which kernel runs the FP32 ring step (Eq. Delta2map) of the
 * tensor-core forms.  Two kernels exist: a register-FFT kernel for even rings
 * whose half-length N is a power of two in [256, 4096] (direct transform) or
 * at most 2048 (Bluestein's algorithm with a power-of-two length), and the
 * shared-memory mixed-radix kernel for any ring.  mode 0 (default): the
 * register kernel for the rings it runs with Bluestein's algorithm, the
 * shared-memory kernel for the others; mode 1: the shared-memory kernel for
 * every ring; mode 2: the register kernel for every ring it can run.  The
 * kernels round differently (each within the form's tolerance), so maps
 * differ in the last bits between modes.  SHT_EINVAL for a NULL plan or
 * another mode. */
int sht_debug_ring_kernel(sht_plan_t plan, int mode);

/* Orders of the tensor-core forms' Delta that can be nonzero, per ring (no
 * counterpart in the paper; it follows from the evanescent skip below): out
 * (host, nrings entries) receives for ring r the limit M_r such that every
 * recurrence value lambda_lm(theta_r) / C_l at orders m >= M_r, l <= lmax,
 * is below the FP32 range (rounds to zero in the precision forms), so that
 * Delta_m(theta_r) is exactly zero there.  The Legendre launches of those
 * forms skip the (m, ring block) items whose order is past every ring of the
 * block, and the FP32 ring kernels read only m < M_r.  mmax + 1 for every
 * ring while the skip is disabled.  Builds the skip tables if needed (one
 * FP64 pass over the recurrence, synchronous).  SHT_EINVAL for a NULL plan or
 * array. */
int sht_order_limits(sht_plan_t plan, int *out);

/* Test hook: overwrite the plan's Delta workspace with 0xFF bytes (NaN in
 * FP32 and FP64) and synchronise the device.  The tensor-core forms leave
 * unwritten the Delta entries that are exactly zero past a ring's last
 * nonzero order, and the ring kernels must not read them: after this call a
 * kernel that did would put NaN into the maps.  No effect before the first
 * transform (no workspace yet).  SHT_EINVAL for a NULL plan. */
int sht_debug_poison_delta(sht_plan_t plan);

/* Evanescent skip of the tensor-core forms (on by default).  For large m
 * near the poles lambda_lm is far below the FP32 range for many degrees (the
 * region below the turning point, where Algorithm 2's rescaling keeps the
 * recurrence alive); those values convert to exact zeros.  With the skip on,
 * the first tensor-core launch of a plan runs one FP64 pass over the
 * recurrence (synchronous) that finds, for every (m, block of 128 ring pairs),
 * the first 64-degree group holding a value representable in FP32 and stores
 * every ring's recurrence state there (about 20 bytes per (m, ring pair));
 * later launches start each work item at that group.  Either way the first
 * tensor-core launch after a change of this setting also builds the plan's
 * per-CTA work lists for it on the host (synchronous), balancing the
 * degrees left in each item.  The maps are
 * bit-identical with the skip on or off (rescaling by powers of two is exact
 * and the skipped values are zeros); the work saved is about 22 % at lmax
 * 2048 on a HEALPix Nside 1024 grid.  enable = 0 turns it off. */
int sht_skip_evanescent(sht_plan_t plan, int enable);

/* Autotuner: pick this plan's tile shapes for form prec and batches of
 * nbatch maps by timing every candidate on the plan's own grid (synthetic
 * zero input in the plan's workspace, CUDA events on `stream`, one untimed
 * launch each), and keep the fastest.  Tunes, for the tensor-core forms, the
 * FP32 ring step's maps per CTA for the smooth and Bluestein ring lists
 * ({1, 2, 4} x {1, 2}) and threads per CTA ({256, 512}); for SHT_FP64, the
 * Legendre step's maps per CTA ({1, 2, 4, 8}, timed on up to 8 maps) and the
 * ring step's maps per CTA ({2, 4, 8, 16}).  The transforms' results do not
 * depend on the tile shapes (every product and fused multiply-add is
 * explicitly rounded), only their speed.  Blocks until done (well under a
 * second for the ring candidates; the FP64 Legendre candidates take about
 * 4 x the time of an 8-map FP64 Legendre launch).  Allocates and frees a
 * temporary map buffer (and, for SHT_FP64, a coefficient buffer) and may grow
 * the plan's workspace.  Not to be called during stream capture.  Errors:
 * SHT_EINVAL (no plan, unknown prec, nbatch < 1), SHT_ENOMEM, SHT_ECUDA. */
int sht_autotune(sht_plan_t plan, int prec, int nbatch, void *stream);

/* Current tile shapes of the plan: out[0..min(n, 6)) = {FP32 ring maps per
 * CTA (smooth list), (Bluestein list), FP32 ring threads per CTA, FP64
 * Legendre maps per CTA, FP64 ring maps per CTA, FP32 ring-analysis maps per
 * CTA of the tensor-core transpose}.  Errors: SHT_EINVAL. */
int sht_tiles(sht_plan_t plan, int *out, int n);

/* Set the first n (0..6) tile shapes, in the order of sht_tiles (e.g. ones an
 * earlier sht_autotune picked and the caller saved).  Each value must be one
 * of the candidates ({1, 2, 4}, {1, 2}, {256, 512}, {1, 2, 4, 8},
 * {1, 2, 4, 8, 16}, {1, 2, 4, 8}), else SHT_EINVAL and nothing changes. */
int sht_set_tiles(sht_plan_t plan, const int *vals, int n);

/* FP64 alm2map that allocates nothing (the paper has no counterpart: this is
 * an interface for callers that must not allocate device memory once their
 * processing loop runs, e.g. a host framework that has reserved nearly all
 * device memory for its own pool, or a latency-critical pipeline in which an
 * allocation after start-up is not acceptable).  Same arguments and result as
 * sht_alm2map_batch(plan, nbatch, alm_dev, map_dev, SHT_FP64, stream), but the
 * Delta_m scratch lives in a 16 MiB array that the library reserves statically
 * on every GPU that loads it, for the life of the process; the call allocates
 * no device memory and calls no cudaMalloc, cudaFree or other allocating CUDA
 * or PyTorch routine (a rejected call only records its error message, like
 * every libsht call).  The plan itself is created (and allocates its tables)
 * beforehand with sht_plan.
 * Limit: nbatch * nrings * (mmax + 1) <= 1,048,576 (16 MiB of complex128), else
 * SHT_EUNSUPPORTED.  The first call on a device looks up the scratch array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  All calls on a device share the one scratch array: calls
 * that overlap on the GPU (different streams, no ordering) race and corrupt
 * each other's results.  The scratch keeps the last call's contents; every
 * entry a call reads is first written by that call. */
int sht_alm2map_noalloc(sht_plan_t plan, int nbatch, const void *alm_dev, void *map_dev, void *stream);

/* Spin-2 (polarisation) synthesis, SHT_FP64 only; not in the paper (its
 * transform extended to the CMB's Q/U field).  Q + i U = -sum_{l>=2}
 * sum_{|m|<=l} (E_lm + i B_lm) 2Y_lm with the spin-weighted harmonics
 * 2Y_lm = ð ð Y_lm / K_l, K_l = sqrt((l-1) l (l+1) (l+2)), ð f = -(sin t)^s
 * (d/dt + (i/sin t) d/dphi)((sin t)^-s f) on spin-s quantities, Y_lm as in
 * sht_alm2map (Condon-Shortley), E_{l,-m} = (-1)^m conj(E_lm) and B alike.
 * elm_dev, blm_dev: nbatch x nalm complex128 each (layout of sht_alm2map;
 * entries with l < 2 and Im of m = 0 are ignored); map_dev: nbatch x 2 x npix
 * float64, map b's Q then its U.  Each map's Q and U go through the ring step
 * of sht_alm2map as two real syntheses of Delta_m^Q = -sum_l (E F1 + i B F2),
 * Delta_m^U = -sum_l (B F1 - i E F2), F1, F2 the half sum and half difference
 * of the spin +2 and -2 functions, built from the scalar recurrence (Eq.
 * assLegRec) and its derivative relation.  Every ring needs sin(theta) > 0
 * (SHT_EUNSUPPORTED otherwise); the accuracy near the poles is limited by
 * cancellation of terms of size l^2 / sin^2(theta) (relative 1e-11 at the
 * first HEALPix ring of nside 1024).  Errors: SHT_EINVAL, SHT_EUNSUPPORTED,
 * SHT_ENOMEM, SHT_ECUDA. */
int sht_alm2map_spin2(sht_plan_t plan, int nbatch, const void *elm_dev, const void *blm_dev, void *map_dev, int prec,
                      void *stream);

/* alm2map of coefficients in host memory into maps in host memory: nsteps
 * batches of nbatch maps, batch k read from alm_host[k] (nbatch x nalm
 * complex128, m-major packed) and written to map_host[k] (nbatch x npix,
 * float64 for SHT_FP64, float32 otherwise), as a caller streaming batches
 * through the GPU would.  The library pipelines the steps (Eq. alm2mapDef per
 * batch, as sht_alm2map_batch): batch k + 1's coefficients go up on one copy
 * stream and batch k - 1's maps come down on another while batch k is
 * transformed on `stream`, through two device buffer sets the plan allocates
 * on first use and keeps (2 nbatch (16 nalm + npix x element size) bytes).
 * The same host array may appear at several steps (each step's copies
 * complete before the next use of its buffer).  Host arrays should be page-
 * locked (cudaHostRegister / cudaMallocHost) for the copies to overlap.
 * Synchronous: returns once every map is in host memory.  Errors: SHT_EINVAL
 * (NULL plan or pointer, nsteps or nbatch < 0, unknown precision),
 * SHT_ENOMEM, SHT_ECUDA, and those of sht_alm2map_batch. */
int sht_alm2map_host(sht_plan_t plan, int nsteps, int nbatch, const void *const *alm_host, void *const *map_host,
                     int prec, void *stream);

/* ---- One transform split over several parts (GPUs): Algorithm 3 (sec.
 * 2.2.3).  The orders m are partitioned for the Legendre step, every part
 * sends each other part the Delta_m(ring) of its orders on that part's rings
 * (one all-to-all exchange, the caller's: e.g. NCCL all_to_all between GPUs,
 * or device copies between parts on one GPU), and the rings are partitioned
 * for the ring step.  Each part's arithmetic is the unpartitioned FP64
 * path's, so the assembled maps equal sht_alm2map_batch's bit for bit.
 * Layouts (complex128, nbatch maps): the send buffer of part p is, for each
 * destination q in order, the rows of q's rings (ascending) x maps x p's
 * orders (ascending): nrings x nbatch x |M_p| entries; the receive buffer of
 * part q is, for each source p in order, q's rings x maps x p's orders:
 * |R_q| x nbatch x (mmax + 1) entries.  The block p -> q has |R_q| x nbatch x
 * |M_p| entries in both. */

/* Host only (no GPU): a balanced partition of orders and rings over nparts.
 * Orders go in pairs (m, mmax - m), whose recurrence lengths lmax - m + 1 sum
 * to a constant when lmax = mmax (the load balancing the paper's conclusion
 * calls for), each pair to the part with the least work so far; rings go in
 * contiguous ranges of about equal pixel count (nphi[r] pixels per ring).
 * Writes m_owner[0..mmax] and ring_owner[0..nrings) in [0, nparts).
 * SHT_EINVAL for bad sizes or NULL arrays. */
int sht_partition(int lmax, int mmax, int nrings, const int *nphi, int nparts, int *m_owner, int *ring_owner);
/* Pixels per ring of the plan (host array of sht_nrings entries). */
int sht_ring_lengths(sht_plan_t plan, int *nphi);
/* Legendre step of part `part` (SHT_FP64 only): Delta_m of every ring for the
 * orders m with m_owner[m] == part, from alm_dev (nbatch x nalm complex128;
 * only those orders are read), into send_dev in the send layout above.
 * m_owner, ring_owner: host arrays as sht_partition writes them.  Uploads its
 * index tables synchronously (after the work already queued on stream).  Errors: SHT_EINVAL, SHT_EUNSUPPORTED (another
 * precision), SHT_ENOMEM, SHT_ECUDA. */
int sht_alm2map_mpart(sht_plan_t plan, int nbatch, int nparts, const int *m_owner, const int *ring_owner, int part,
                      const void *alm_dev, void *send_dev, int prec, void *stream);
/* Ring step of part `part` (SHT_FP64 only): from recv_dev (the receive layout
 * above, every order of every ring with ring_owner[r] == part), the pixels of
 * those rings in map_dev (nbatch x npix float64; other rings untouched).  The
 * orders are gathered into the plan's workspace (grown as needed), then the
 * ring kernels run over the part's rings.  Errors as sht_alm2map_mpart. */
int sht_ring_synth_part(sht_plan_t plan, int nbatch, int nparts, const int *m_owner, const int *ring_owner, int part,
                        const void *recv_dev, void *map_dev, int prec, void *stream);

/* Many requests of different grids and band limits (one map each) in one
 * call: the batching form.  Request i transforms alm_dev[i] (plans[i]'s
 * nalm complex128) into map_dev[i] (plans[i]'s npix reals).  FP64: the
 * Legendre step of all requests runs as one persistent launch whose CTAs
 * take (request, m, ring block) work items, sorted by decreasing cost, from
 * an atomic counter, then one launch per ring list does all rings; the
 * context is capturable in a CUDA graph (no allocation or host sync inside
 * sht_multi_alm2map; pointers are kernel parameters, so a captured graph
 * replays with the pointers it was captured with).  Tensor-core forms: one
 * operand-prep launch over all requests' (request, m) items, then one persistent
 * tensor-core Legendre launch over all requests' (request, m, ring block)
 * items (one CTA per SM; each CTA runs a fixed list: the items, longest
 * first, each given to the CTA with the least work so far), then one
 * FP32 ring launch per ring list; equally capturable.  Creating a tensor-core
 * context builds each plan's operand buffer and skip tables (synchronous);
 * while the context runs, the plans' own transforms must not run concurrently
 * (they share those buffers); a bounded device wait that runs out is reported
 * by sht_sync(plans[0]).  A plan may appear more than once (requests of
 * equal grid and band limit): in the tensor-core forms every repeat gets its
 * own operand buffer, allocated by sht_multi_create (tc operand bytes of that
 * plan each).  1 <= nreq <= 256; all plans on one device; the plans must
 * outlive the context.
 * sht_alm2map_multi = create + run + stream synchronize + destroy. */
typedef struct sht_multi_s *sht_multi_t;
int sht_multi_create(int nreq, const sht_plan_t *plans, int prec, sht_multi_t *out);
int sht_multi_alm2map(sht_multi_t multi, const void *const *alm_dev, void *const *map_dev, void *stream);
int sht_multi_destroy(sht_multi_t multi);

/* Tile shapes of a multi-request context (no counterpart in the paper;
 * results do not depend on them): vals[0] = persistent CTAs per SM of the
 * FP64 Legendre launch (1..32, default 8), vals[1] = threads per CTA of the
 * tensor-core forms' shared-memory ring kernel (256 or 512, default 256).
 * n >= 2.  SHT_EINVAL for a NULL context or array, n < 2 or a value out of
 * range. */
int sht_multi_tiles(sht_multi_t multi, int *out, int n);
int sht_multi_set_tiles(sht_multi_t multi, const int *vals, int n);

/* Autotuner of a multi-request context: times each candidate (FP64: 2, 4, 8,
 * 16 CTAs per SM; tensor-core forms: 256 or 512 ring threads) on the caller's
 * requests (one untimed call, one call timed with events on `stream`) and
 * keeps the fastest.  The maps hold the last call's result.  Synchronises
 * `stream`.  Errors as sht_multi_alm2map. */
int sht_multi_autotune(sht_multi_t multi, const void *const *alm_dev, void *const *map_dev, void *stream);

/* Test hook: sht_debug_poison_delta for the Delta workspace of a
 * multi-request context.  SHT_EINVAL for a NULL context. */
int sht_multi_debug_poison_delta(sht_multi_t multi);
int sht_alm2map_multi(int nreq, const sht_plan_t *plans, const void *const *alm_dev, void *const *map_dev,
                      int prec, void *stream);

/* Message describing the last error on the calling thread ("" if none). */
const char *sht_last_error(void);

/* Per-stage GPU timing (the paper times its kernels with gettimeofday,
 * sec. 6; here CUDA events are recorded on the launch stream around every
 * kernel the plan launches while profiling is enabled).
 * Stages: SHT_STAGE_LEGENDRE (Legendre step), SHT_STAGE_RING (ring step),
 * SHT_STAGE_ADJ_RING, SHT_STAGE_ADJ_LEGENDRE (the transpose's two steps),
 * SHT_STAGE_OPERAND_PREP (the tensor-core forms' conversion of a_lm into the
 * split B operand, before each Legendre launch).
 * sht_profile_read synchronises the plan's device, writes the summed
 * milliseconds and the launch count of each of the first nstage stages into
 * ms[] and launches[] (either may be NULL) and resets the counters. */
#define SHT_STAGE_LEGENDRE 0
#define SHT_STAGE_RING 1
#define SHT_STAGE_ADJ_RING 2
#define SHT_STAGE_ADJ_LEGENDRE 3
#define SHT_STAGE_OPERAND_PREP 4
#define SHT_NSTAGES 5
int sht_profile(sht_plan_t plan, int enable);
int sht_profile_read(sht_plan_t plan, int nstage, double *ms, long long *launches);

/* Wait for all work on the plan's device and report device-side failures:
 * SHT_ETIMEOUT if a kernel of this plan gave up a bounded wait (the kernel
 * then returned early and its output is invalid; the flag is cleared),
 * SHT_ECUDA for a CUDA error, else SHT_OK. */
int sht_sync(sht_plan_t plan);

/* Test hook for the bounded device-side waits: the next tensor-core Legendre
 * launch of this plan (per-call or cached-Lambda form) skips, in its CTA 0,
 * the operand copies of stage number `stage` (counted over that CTA's work
 * items; -1 clears the hook).  The MMA warp's wait for that stage then runs
 * out after its 2 s limit; the CTA stops, drains (bounded) what it issued,
 * frees its tensor memory and sets the plan's status word, so sht_sync
 * reports SHT_ETIMEOUT and that launch's output is invalid.  No fault, trap or
 * endless wait is involved; the context stays usable.  Errors: SHT_EINVAL. */
int sht_debug_withhold_stage(sht_plan_t plan, int stage);

/* Number of kernels libsht has launched in this process (all plans). */
unsigned long long sht_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* SHT_H */
