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

#include <stddef.h>

#include "wolff.h"
#include "wolff_internal.h"

using namespace wolff;

namespace {

// Control block, then the cluster list of up to WOLFF_STATIC_MAX_SITES entries.
constexpr size_t kScratchBytes =
    sizeof(DevCtl) + (size_t)WOLFF_STATIC_MAX_SITES * sizeof(uint32_t);
// the size the header states: 1 KiB of control block and 4 MiB of list
static_assert(sizeof(DevCtl) == 1024, "the header states a 1 KiB control block");
static_assert(kScratchBytes == (4u << 20) + 1024u, "the header states 4 MiB + 1 KiB");

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Device address of the scratch array on the current device.  In host code
// the symbol's name is only a host-side stand-in, so the address is asked of
// the runtime with the device current.  It is looked up on every call: the
// lookup is cheap next to the launches, and a cached address would go stale
// if the caller reset the device (the module, and the array with it, can
// move when it is loaded again).
cudaError_t scratch_for_current_device(void **out) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return e;
    *out = ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" wolff_status wolff_step_static(int dim, int L, double J, double T, uint64_t seed,
                                          uint64_t t0, uint64_t n_updates, void *d_spins,
                                          void *d_records, void *stream) {
    // ---- everything that can be rejected is checked before the lattice is
    // touched, so a rejected call leaves the caller's buffer as it was
    const bool shape = (dim == 2 && L >= 2 && L <= 32767) || (dim == 3 && L >= 2 && L <= 1024);
    if (!shape || !(J >= 0.0) || !(T > 0.0) || !d_spins) return WOLFF_EINVAL;
    uint64_t n = 1;
    for (int d = 0; d < dim; ++d) n *= (uint64_t)L;
    if (n > WOLFF_STATIC_MAX_SITES) return WOLFF_EINVAL;
    // the 32-sites-per-thread recount reads the lattice in 16-byte vectors
    if (reinterpret_cast<uintptr_t>(d_spins) % 16u) return WOLFF_EINVAL;
    if (d_records && reinterpret_cast<uintptr_t>(d_records) % alignof(wolff_record))
        return WOLFF_EINVAL;

    void *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return WOLFF_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int device = 0, sms = 0;
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return WOLFF_ECUDA;
    const int threads = 256;
    int blocks = 0;
    if (n_updates) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel(dim), threads,
                                                          0) != cudaSuccess)
            return WOLFF_ECUDA;
        blocks = (int)(n / 2048u);
        if (blocks < 1) blocks = 1;
        if (blocks > sms) blocks = sms;
        if (blocks > per_sm * sms) blocks = per_sm * sms;
        if (blocks < 1) return WOLFF_EUNSUPPORTED;
    }

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
    if (e != cudaSuccess) return WOLFF_ECUDA;
    // an entry other than +-1 becomes -1 and latches WOLFF_EINVAL, which the
    // update kernel sees before its first update: it then runs none
    e = launch_from_pm1(p.spins, static_cast<const int8_t *>(d_spins), p.g.N, p.ctl, s);
    if (e != cudaSuccess) return WOLFF_ECUDA;
    // from here on the lattice holds spin bytes: whatever fails, the
    // conversion back to +-1 is still enqueued
    e = launch_measure_full(dim, p.spins, p.g, p.ctl, 1, s);
    // the update expects every cluster-list slot to hold the empty marker
    if (e == cudaSuccess) e = cudaMemsetAsync(p.list, 0xFF, (size_t)p.g.N * sizeof(uint32_t), s);
    if (e == cudaSuccess && n_updates) {
        void *args[] = {&p};
        e = cudaLaunchCooperativeKernel(persistent_kernel(dim), dim3(blocks), dim3(threads), args,
                                        0, s);
    }
    const cudaError_t back = launch_to_pm1(static_cast<int8_t *>(d_spins), p.spins, p.g.N, s);
    return (e == cudaSuccess && back == cudaSuccess) ? WOLFF_OK : WOLFF_ECUDA;
}

extern "C" wolff_status wolff_step_static_status(void *stream, int *device_status,
                                                 uint32_t *detail, uint64_t *t_next) {
    void *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return WOLFF_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DevCtl h;
    cudaError_t e = cudaMemcpyAsync(&h, scratch, sizeof(DevCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return WOLFF_ECUDA;
    if (device_status) *device_status = (int)h.status;
    if (detail) *detail = h.err_detail;
    if (t_next) *t_next = h.t;
    return WOLFF_OK;
}
