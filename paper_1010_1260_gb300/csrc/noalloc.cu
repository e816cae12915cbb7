// sht_alm2map_noalloc: the FP64 alm2map with its scratch in a fixed,
// statically allocated device array instead of the plan's workspace.
//
// Who needs this: callers that must not allocate device memory once their
// processing loop is running -- for example a host framework that has
// reserved (nearly) all device memory for its own pool, so that a
// cudaMalloc from a library would fail, or a latency-critical pipeline in
// which an allocation (which can synchronise the device) is not acceptable
// after start-up.  They create the plan during set-up and then call this
// entry point, which allocates nothing.
//
// The scratch is the Delta_m(ring) array that the Legendre step writes and
// the ring step reads.  It lives in the file-scope array below, which every
// GPU that loads the library holds until the process exits.  Host code must
// not pass the array's name to a kernel (in host code it is only a stand-in
// for the symbol); its device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
#include "sht.h"
#include "sht_internal.cuh"

#include <mutex>

namespace sht {
const DevPlan *plan_dev(sht_plan_t p);
void plan_fp64_tiles(sht_plan_t p, int *bc, int *ring_g);
int plan_device(sht_plan_t p);
std::mutex *plan_mutex(sht_plan_t p);
int record_error(int code, const char *msg);
int record_cuda_error(cudaError_t e, const char *what);
void clear_error();
void count_launch();
}  // namespace sht

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr size_t kScratchElems = kScratchBytes / sizeof(double2);

static __device__ __align__(256) double2 g_noalloc_scratch[kScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double2 *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up on first use).
int scratch_on_current_device(double2 **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return sht::record_cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return sht::record_error(SHT_EUNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return sht::record_cuda_error(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_ptr[dev] = static_cast<double2 *>(ptr);
    }
    *out = g_scratch_ptr[dev];
    return SHT_OK;
}

}  // namespace

extern "C" int sht_alm2map_noalloc(sht_plan_t plan, int nbatch, const void *alm_dev, void *map_dev,
                                   void *stream)
{
    sht::clear_error();
    if (!plan) return sht::record_error(SHT_EINVAL, "null plan");
    if (nbatch < 0) return sht::record_error(SHT_EINVAL, "nbatch < 0");
    if (nbatch == 0) return SHT_OK;
    if (!alm_dev || !map_dev) return sht::record_error(SHT_EINVAL, "null device pointer");
    const sht::DevPlan &P = *sht::plan_dev(plan);
    const size_t need = (size_t)nbatch * P.nrings * (size_t)(P.mmax + 1);
    if (need > kScratchElems)
        return sht::record_error(SHT_EUNSUPPORTED,
                                 "sht_alm2map_noalloc: nbatch * nrings * (mmax + 1) exceeds the 16 MiB "
                                 "static scratch (1048576 complex entries)");
    if (nbatch > 32768) return sht::record_error(SHT_EUNSUPPORTED, "nbatch > 32768");

    std::lock_guard<std::mutex> lk(*sht::plan_mutex(plan));
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return sht::record_cuda_error(e, "cudaGetDevice");
    const int dev = sht::plan_device(plan);
    if (prev != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return sht::record_cuda_error(e, "cudaSetDevice");
    double2 *scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc == SHT_OK) {
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        // The Legendre step writes every (ring, m) entry of the scratch that
        // the ring step reads, so nothing has to be cleared between calls.
        // The plan's tile shapes (sht_autotune) apply here as in sht_alm2map_batch.
        int bc = 0, rg = 0;
        sht::plan_fp64_tiles(plan, &bc, &rg);
        e = sht::launch_legendre_fwd_fp64(P, static_cast<const double2 *>(alm_dev), scratch, nbatch, bc, st);
        if (e == cudaSuccess) {
            sht::count_launch();
            e = sht::launch_ring_synth_fp64(P, scratch, static_cast<double *>(map_dev), nbatch, rg, st);
            if (e == cudaSuccess)
                for (int i = 0; i < sht::ring_launches(P); ++i) sht::count_launch();
        }
        if (e != cudaSuccess) rc = sht::record_cuda_error(e, "sht_alm2map_noalloc launch");
    }
    if (prev != dev) cudaSetDevice(prev);
    return rc;
}
