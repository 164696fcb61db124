// wolff_probe.cu -- L2 bandwidth probe (a measurement aid; the paper has no
// counterpart).
//
// The update's working set (one spin byte per site and the touched part of
// the cluster list, 16.8 MB + a few MB on the 2^24-site lattices) lives in
// the 129 MB L2, so the memory roofline of the growth kernels has an L2 side
// as well as the HBM one.  Its denominator is measured here: every thread of
// a full-occupancy grid streams a buffer that fits in L2 with 16-byte loads
// that skip L1 (ld.global.cg), `passes` times in one launch; mode 1 also
// writes each vector back (a read-modify-write stream).  Timed on the host
// with CUDA events, bytes moved / time is the L2 bandwidth the SMs can draw.
#include <cuda_runtime.h>

#include "wolff.h"

namespace {

__global__ void k_l2_stream(uint4 *buf, unsigned long long n16, int passes, int mode,
                            unsigned int *sink) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned int acc = 0;
    for (int p = 0; p < passes; ++p) {
        for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
             k < n16; k += stride) {
            uint4 v = __ldcg(buf + k);
            // a running hash of every loaded word (not an XOR, which two
            // passes over the same data would cancel): the loads stay live
            acc = acc * 31u + (v.x ^ v.y ^ v.z ^ v.w);
            if (mode == 1) {
                v.x += 1u;
                __stcg(buf + k, v);
            }
        }
    }
    if (acc == 0x2545F491u) sink[0] = acc;   // practically never taken
}

}  // namespace

extern "C" wolff_status wolff_l2_probe(void *d_buf, size_t bytes, int passes, int mode,
                                       uint32_t *d_sink, void *stream) {
    if (!d_buf || !d_sink || bytes < 16 || bytes % 16u || passes < 1 || passes > 100000 ||
        (mode != 0 && mode != 1) || reinterpret_cast<uintptr_t>(d_buf) % 16u ||
        reinterpret_cast<uintptr_t>(d_sink) % 4u)
        return WOLFF_EINVAL;
    int device = 0, sms = 0, per_sm = 0;
    const int threads = 256;
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_l2_stream, threads, 0) !=
            cudaSuccess)
        return WOLFF_ECUDA;
    if (per_sm < 1) per_sm = 1;
    const unsigned long long n16 = bytes / 16u;
    unsigned long long blocks = (unsigned long long)sms * (unsigned long long)per_sm;
    const unsigned long long need = (n16 + threads - 1) / threads;
    if (blocks > need) blocks = need;
    k_l2_stream<<<(unsigned)blocks, threads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        static_cast<uint4 *>(d_buf), n16, passes, mode, d_sink);
    return cudaGetLastError() == cudaSuccess ? WOLFF_OK : WOLFF_ECUDA;
}
