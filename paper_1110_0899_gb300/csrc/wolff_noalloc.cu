// wolff_noalloc.cu -- wolff_step_static: the Wolff update without any
// device allocation.
//
// Who needs this.  Some callers cannot call cudaMalloc at the point where
// they want to run updates: code embedded in a framework whose caching
// allocator has already reserved the device memory (a stray cudaMalloc then
// fails or fragments the pool), latency-critical loops where cudaMalloc's
// implicit device-wide synchronisation is not acceptable, and programs that
// must fix their whole device-memory budget when the library is loaded.
// ising_init either allocates the workspace or asks the caller for one; this
// entry point needs neither: its scratch (the control block and the cluster
// list) lives in the file-scope array below, which every GPU that loads the
// library holds until the process exits.
//
// The kernel is the persistent update of wolff_kernels.cu, launched on the
// static scratch instead of a context's workspace.
#include <cuda_runtime.h>

#include <mutex>

#include "wolff.h"
#include "wolff_internal.h"

using namespace wolff;

namespace {

// Control block, then the cluster list of up to WOLFF_STATIC_MAX_SITES entries.
constexpr size_t kScratchBytes =
    sizeof(DevCtl) + (size_t)WOLFF_STATIC_MAX_SITES * sizeof(uint32_t);

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The symbol's
// name in host code is only a host-side stand-in, so its device address is
// looked up once per device, with that device current.
cudaError_t scratch_for_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" wolff_status wolff_step_static(int dim, int L, double J, double T, uint64_t seed,
                                          uint64_t t0, uint64_t n_updates, void *d_spins,
                                          void *d_records, void *stream) {
    const bool shape = (dim == 2 && L >= 2 && L <= 32767) || (dim == 3 && L >= 2 && L <= 1024);
    if (!shape || !(J >= 0.0) || !(T > 0.0) || !d_spins) return WOLFF_EINVAL;
    uint64_t n = 1;
    for (int d = 0; d < dim; ++d) n *= (uint64_t)L;
    if (n > WOLFF_STATIC_MAX_SITES) return WOLFF_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_spins) % 4u) return WOLFF_EINVAL;

    void *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return WOLFF_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int device = 0, sms = 0;
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return WOLFF_ECUDA;

    StepParams p = {};   // fields this path does not use stay zero
    p.ctl = static_cast<DevCtl *>(scratch);
    p.list = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + sizeof(DevCtl));
    // the caller's int8 +-1 lattice is turned into the kernel's spin bytes in
    // place and back again at the end
    p.spins = static_cast<uint8_t *>(d_spins);
    p.records = static_cast<wolff_record *>(d_records);
    p.g.L = (uint32_t)L;
    p.g.N = (uint32_t)n;
    p.g.LL = (uint32_t)L * (uint32_t)L;
    p.key0 = (uint32_t)seed;
    p.key1 = (uint32_t)(seed >> 32);
    p.thr = wolff_bond_threshold(J, T);
    p.t0 = t0;
    p.n = n_updates;
    p.wait_ns = 2000000000ull;
    p.t_up = 512;
    p.t_down = 256;
    p.win_levels = 0;
    p.budget_ns = 0;
    p.q = 2;

    // every call starts from a cleared control block: the array keeps the
    // previous call's contents
    cudaError_t e = launch_reset_ctl(p.ctl, t0, s);
    if (e == cudaSuccess)
        e = launch_from_pm1(p.spins, static_cast<const int8_t *>(d_spins), p.g.N, p.ctl, s);
    if (e == cudaSuccess) e = launch_measure_full(dim, p.spins, p.g, p.ctl, 1, s);
    // the update expects every cluster-list slot to hold the empty marker
    if (e == cudaSuccess) e = cudaMemsetAsync(p.list, 0xFF, (size_t)p.g.N * sizeof(uint32_t), s);
    if (e == cudaSuccess && n_updates) {
        const int threads = 256;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel(dim),
                                                          threads, 0);
        int blocks = (int)(p.g.N / 2048u);
        if (blocks < 1) blocks = 1;
        if (blocks > sms) blocks = sms;
        if (e == cudaSuccess && blocks > per_sm * sms) blocks = per_sm * sms;
        if (e == cudaSuccess && blocks < 1) return WOLFF_EUNSUPPORTED;
        void *args[] = {&p};
        if (e == cudaSuccess)
            e = cudaLaunchCooperativeKernel(persistent_kernel(dim), dim3(blocks), dim3(threads),
                                            args, 0, s);
    }
    if (e == cudaSuccess)
        e = launch_to_pm1(static_cast<int8_t *>(d_spins), p.spins, p.g.N, s);
    return e == cudaSuccess ? WOLFF_OK : WOLFF_ECUDA;
}
