// wolff_kernels.cu -- sm_103a kernels of the Wolff single-cluster update.
//
// Two schedules of the same level-synchronous growth (section 4, step (iii')):
//   persistent: one cooperative launch runs every update of a wolff_step;
//     levels are separated by a bounded grid barrier (the paper's
//     quasi-block synchronisation, section 3, is replaced by an
//     acquire/release generation barrier over co-resident CTAs);
//   graph: one kernel launch per level inside a conditional WHILE node, the
//     launch boundary being the barrier, nested in a WHILE node over updates.
// Both append newly claimed sites to the cluster list with one atomic per
// warp, so level k's frontier is list[lo_k, hi_k) -- the paper's ic/in
// bookkeeping (section 2) without per-direction barriers: the atomic claim
// (flip-on-add, allowed by the freedom in the timing of the flip noted in
// section 2) already prevents double adds.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "wolff_device.cuh"

namespace wolff {

static inline unsigned grid_for(unsigned long long work, unsigned long long cap) {
    unsigned long long b = work < cap ? work : cap;
    return (unsigned)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------------------
// a1: initial lattice from Philox (tag 2)
__global__ void k_init(uint8_t *spins, uint32_t N, uint32_t k0, uint32_t k1) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += gridDim.x * blockDim.x) {
        const Philox4 r = philox4x32_10(i, 0u, 0u, kTagInit, k0, k1);
        spins[i] = (r.v[0] >> 31) ? 0x00 : 0x03;
    }
}

cudaError_t launch_init(uint8_t *spins, Geometry g, uint32_t k0, uint32_t k1,
                        cudaStream_t s) {
    const unsigned blocks = grid_for((g.N + 255) / 256, 4096ull);
    k_init<<<blocks, 256, 0, s>>>(spins, g.N, k0, k1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// L2 warm-up: a lattice evicted from L2 (by other work between calls) would
// make every early access of the update chain a DRAM round trip; streaming
// it once at full bandwidth brings it back.  Each thread touches one 128-byte
// line with a prefetch.
__global__ void k_prefetch_l2(const uint8_t *base, unsigned long long bytes) {
    for (unsigned long long off = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) * 128ull;
         off < bytes; off += (unsigned long long)gridDim.x * blockDim.x * 128ull)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + off));
}

cudaError_t launch_prefetch_l2(const void *base, unsigned long long bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    const unsigned long long lines = (bytes + 127) / 128;
    k_prefetch_l2<<<grid_for((lines + 255) / 256, 2048ull), 256, 0, s>>>(
        static_cast<const uint8_t *>(base), bytes);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a8: full recount.  One CTA per row of L sites (rows along x), threads over
// x; E_bond gets s_i (s_{x+1} + s_{y+1} [+ s_{z+1}]), M gets s_i.
template <int DIM>
__global__ void k_measure_full(const uint8_t *spins, Geometry g, DevCtl *ctl) {
    const uint32_t rows = g.N / g.L;
    long long e = 0, m = 0;
    for (uint32_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const uint32_t y = row % g.L;
        const uint32_t base = row * g.L;
        const uint32_t yup = (y + 1 == g.L) ? base + g.L - g.LL : base + g.L;  // +L with wrap in y
        uint32_t zup = 0;
        if (DIM == 3) {
            const uint32_t z = row / g.L;
            zup = (z + 1 == g.L) ? base + g.LL - g.N : base + g.LL;
        }
        for (uint32_t x = threadIdx.x; x < g.L; x += blockDim.x) {
            const int si = (spins[base + x] & 1) ? 1 : -1;
            const uint32_t xr = (x + 1 == g.L) ? 0 : x + 1;
            int nbsum = ((spins[base + xr] & 1) ? 1 : -1) + ((spins[yup + x] & 1) ? 1 : -1);
            if (DIM == 3) nbsum += (spins[zup + x] & 1) ? 1 : -1;
            e += si * nbsum;
            m += si;
        }
    }
    e = block_sum(e);
    m = block_sum(m);
    if (threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_E), (unsigned long long)e);
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_M), (unsigned long long)m);
    }
}

// ---- 32 sites per thread (L a multiple of 32) ------------------------------
// A word w covers sites 32w .. 32w+31 of one row, bit k = site 32w + k is +1.
// Its forward bonds along x are the bits against the word shifted by one
// (the last site against bit 0 of the next word of the row, wrapping to the
// row's first word); along y (z) the bits of the word L/32 (L^2/32) further
// on, wrapping within the plane (the lattice).  Over the 32 sites the bonds
// sum to 32 - 2 popc(b ^ nb) and the spins to 2 popc(b) - 32.
struct WordGeom {
    uint32_t wpr, plane, words;   // words per row, per xy plane (2D: all), in all
};

__device__ __forceinline__ WordGeom word_geom(const Geometry &g, int dim) {
    WordGeom w;
    w.wpr = g.L >> 5;
    w.words = g.N >> 5;
    w.plane = dim == 3 ? (g.LL >> 5) : w.words;
    return w;
}

template <int DIM>
__device__ __forceinline__ void word_neighbours(const WordGeom &wg, uint32_t w, uint32_t &nxt,
                                                uint32_t &up, uint32_t &zup) {
    const uint32_t wr = w % wg.wpr;
    nxt = (wr + 1 == wg.wpr) ? w - wr : w + 1;
    const uint32_t ip = DIM == 3 ? w % wg.plane : w;
    up = (ip + wg.wpr < wg.plane) ? w + wg.wpr : w + wg.wpr - wg.plane;
    zup = 0;
    if (DIM == 3) zup = (w + wg.plane < wg.words) ? w + wg.plane : w + wg.plane - wg.words;
}

__device__ __forceinline__ int word_bonds(uint32_t b, uint32_t nb) {
    return 32 - 2 * __popc(b ^ nb);
}

// Bit 0 of each of 4 bytes -> 4 bits (byte k -> bit k): the masked bytes
// times 2^24 + 2^17 + 2^10 + 2^3 put byte k's bit at 24 + k with every
// other partial product outside bits 24..27 and no carries.
__device__ __forceinline__ uint32_t bytes_to_nibble(uint32_t w) {
    return (((w & 0x01010101u) * 0x01020408u) >> 24) & 0xFu;
}

// 32 spin bytes (16-byte aligned) -> their bit mask.
__device__ __forceinline__ uint32_t load_word_bits(const uint8_t *p) {
    const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
    const uint4 b = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
    return bytes_to_nibble(a.x) | bytes_to_nibble(a.y) << 4 | bytes_to_nibble(a.z) << 8 |
           bytes_to_nibble(a.w) << 12 | bytes_to_nibble(b.x) << 16 | bytes_to_nibble(b.y) << 20 |
           bytes_to_nibble(b.z) << 24 | bytes_to_nibble(b.w) << 28;
}

// 4 bits -> 4 spin bytes (0x03 for +1, 0x00 for -1): the nibble times
// 1 + 2^7 + 2^14 + 2^21 puts bit k at 8k (partial products at 0-3, 7-10,
// 14-17, 21-24 never overlap), masked and tripled.
__device__ __forceinline__ uint32_t nibble_to_bytes(uint32_t nib) {
    return ((nib * 0x00204081u) & 0x01010101u) * 3u;
}

// a8 with 32 sites per thread: 64 bytes of loads (the word and the one above
// in y; 96 in 3D) and one byte of the next word for 32 sites.
template <int DIM>
__global__ void k_measure_words(const uint8_t *spins, Geometry g, DevCtl *ctl) {
    const WordGeom wg = word_geom(g, DIM);
    long long e = 0, m = 0;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < wg.words;
         w += gridDim.x * blockDim.x) {
        uint32_t nxt, up, zup;
        word_neighbours<DIM>(wg, w, nxt, up, zup);
        const uint32_t b = load_word_bits(spins + 32ull * w);
        const uint32_t right = (b >> 1) | ((uint32_t)(spins[32ull * nxt] & 1u) << 31);
        int bonds = word_bonds(b, right) + word_bonds(b, load_word_bits(spins + 32ull * up));
        if (DIM == 3) bonds += word_bonds(b, load_word_bits(spins + 32ull * zup));
        e += bonds;
        m += 2 * __popc(b) - 32;
    }
    e = block_sum(e);
    m = block_sum(m);
    if (threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_E), (unsigned long long)e);
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_M), (unsigned long long)m);
    }
}

__global__ void k_zero_full(DevCtl *ctl) {
    ctl->full_E = 0;
    ctl->full_M = 0;
}

__global__ void k_full_to_chain(DevCtl *ctl) {
    ctl->E = ctl->full_E;
    ctl->M = ctl->full_M;
}

// Blocks for the 32-sites-per-thread passes: enough 256-thread blocks for
// the words, at most 4 per SM of a 152-SM GPU (one pair of atomics each).
static inline unsigned word_blocks(const Geometry &g) {
    return grid_for(((g.N >> 5) + 255ull) / 256ull, 608ull);
}

cudaError_t launch_measure_full(int dim, const uint8_t *spins, Geometry g, DevCtl *ctl,
                                int set_chain, cudaStream_t s) {
    k_zero_full<<<1, 1, 0, s>>>(ctl);
    if (g.L % 32 == 0) {
        if (dim == 2)
            k_measure_words<2><<<word_blocks(g), 256, 0, s>>>(spins, g, ctl);
        else
            k_measure_words<3><<<word_blocks(g), 256, 0, s>>>(spins, g, ctl);
    } else {
        const uint32_t rows = g.N / g.L;
        const unsigned blocks = grid_for(rows, 8192ull);
        const unsigned threads = g.L >= 256 ? 256 : 64;
        if (dim == 2)
            k_measure_full<2><<<blocks, threads, 0, s>>>(spins, g, ctl);
        else
            k_measure_full<3><<<blocks, threads, 0, s>>>(spins, g, ctl);
    }
    if (set_chain) k_full_to_chain<<<1, 1, 0, s>>>(ctl);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// state conversion (checkpoint / restore)
__global__ void k_from_pm1(uint8_t *spins, const int8_t *src, uint32_t N, DevCtl *ctl) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += gridDim.x * blockDim.x) {
        const int v = src[i];
        if (v == 1) {
            spins[i] = 0x03;
        } else if (v == -1) {
            spins[i] = 0x00;
        } else {
            spins[i] = 0x00;
            raise_status(ctl, WOLFF_EINVAL, i);
        }
    }
}

__global__ void k_to_pm1(int8_t *dst, const uint8_t *spins, uint32_t N) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += gridDim.x * blockDim.x)
        dst[i] = (spins[i] & 1) ? 1 : -1;
}

// Upload path in one pass: converts an int8 +-1 lattice into spin bytes and
// sums E_bond and M from the same input (forward neighbours read from src);
// entries other than +-1 become -1 and latch WOLFF_EINVAL.
template <int DIM>
__global__ void k_from_pm1_measure(uint8_t *spins, const int8_t *src, Geometry g, DevCtl *ctl) {
    const uint32_t rows = g.N / g.L;
    long long e = 0, m = 0;
    for (uint32_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const uint32_t y = row % g.L;
        const uint32_t base = row * g.L;
        const uint32_t yup = (y + 1 == g.L) ? base + g.L - g.LL : base + g.L;
        uint32_t zup = 0;
        if (DIM == 3) {
            const uint32_t z = row / g.L;
            zup = (z + 1 == g.L) ? base + g.LL - g.N : base + g.LL;
        }
        for (uint32_t x = threadIdx.x; x < g.L; x += blockDim.x) {
            const int v = src[base + x];
            if (v != 1 && v != -1) raise_status(ctl, WOLFF_EINVAL, base + x);
            spins[base + x] = v == 1 ? 0x03 : 0x00;
            const int si = v == 1 ? 1 : -1;
            const uint32_t xr = (x + 1 == g.L) ? 0 : x + 1;
            int nbsum = (src[base + xr] == 1 ? 1 : -1) + (src[yup + x] == 1 ? 1 : -1);
            if (DIM == 3) nbsum += src[zup + x] == 1 ? 1 : -1;
            e += si * nbsum;
            m += si;
        }
    }
    e = block_sum(e);
    m = block_sum(m);
    if (threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_E), (unsigned long long)e);
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_M), (unsigned long long)m);
        // the last block to finish publishes the sums as the chain state
        __threadfence();
        if (atomicAdd(&ctl->up_blocks, 1u) == gridDim.x - 1) {
            __threadfence();
            ctl->E = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_E), 0ull);
            ctl->M = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_M), 0ull);
            ctl->up_blocks = 0;
        }
    }
}

// Bit-packed upload: bit i of word i / 32 set <=> spin +1.  Same single pass
// as k_from_pm1_measure (spin bytes, E_bond and M from the input bits).
__device__ __forceinline__ int bit_spin(const uint32_t *bits, uint32_t i) {
    return ((__ldg(bits + (i >> 5)) >> (i & 31u)) & 1u) ? 1 : -1;
}

template <int DIM>
__global__ void k_from_bits_measure(uint8_t *spins, const uint32_t *bits, Geometry g,
                                    DevCtl *ctl) {
    const uint32_t rows = g.N / g.L;
    long long e = 0, m = 0;
    for (uint32_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const uint32_t y = row % g.L;
        const uint32_t base = row * g.L;
        const uint32_t yup = (y + 1 == g.L) ? base + g.L - g.LL : base + g.L;
        uint32_t zup = 0;
        if (DIM == 3) {
            const uint32_t z = row / g.L;
            zup = (z + 1 == g.L) ? base + g.LL - g.N : base + g.LL;
        }
        for (uint32_t x = threadIdx.x; x < g.L; x += blockDim.x) {
            const int si = bit_spin(bits, base + x);
            spins[base + x] = si > 0 ? 0x03 : 0x00;
            const uint32_t xr = (x + 1 == g.L) ? 0 : x + 1;
            int nbsum = bit_spin(bits, base + xr) + bit_spin(bits, yup + x);
            if (DIM == 3) nbsum += bit_spin(bits, zup + x);
            e += si * nbsum;
            m += si;
        }
    }
    e = block_sum(e);
    m = block_sum(m);
    if (threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_E), (unsigned long long)e);
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_M), (unsigned long long)m);
        __threadfence();
        if (atomicAdd(&ctl->up_blocks, 1u) == gridDim.x - 1) {
            __threadfence();
            ctl->E = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_E), 0ull);
            ctl->M = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_M), 0ull);
            ctl->up_blocks = 0;
        }
    }
}

// The bit-packed upload with 32 sites per thread (L a multiple of 32): one
// word and its neighbour words in, 32 spin bytes out (two 16-byte stores),
// E_bond and M published by the last block as in k_from_bits_measure.
template <int DIM>
__global__ void k_from_bits_words(uint8_t *spins, const uint32_t *bits, Geometry g,
                                  DevCtl *ctl) {
    const WordGeom wg = word_geom(g, DIM);
    long long e = 0, m = 0;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < wg.words;
         w += gridDim.x * blockDim.x) {
        uint32_t nxt, up, zup;
        word_neighbours<DIM>(wg, w, nxt, up, zup);
        const uint32_t b = __ldg(bits + w);
        const uint32_t right = (b >> 1) | (__ldg(bits + nxt) << 31);
        int bonds = word_bonds(b, right) + word_bonds(b, __ldg(bits + up));
        if (DIM == 3) bonds += word_bonds(b, __ldg(bits + zup));
        e += bonds;
        m += 2 * __popc(b) - 32;
        uint4 *dst = reinterpret_cast<uint4 *>(spins + 32ull * w);
        dst[0] = make_uint4(nibble_to_bytes(b & 0xFu), nibble_to_bytes((b >> 4) & 0xFu),
                            nibble_to_bytes((b >> 8) & 0xFu), nibble_to_bytes((b >> 12) & 0xFu));
        dst[1] = make_uint4(nibble_to_bytes((b >> 16) & 0xFu), nibble_to_bytes((b >> 20) & 0xFu),
                            nibble_to_bytes((b >> 24) & 0xFu), nibble_to_bytes(b >> 28));
    }
    e = block_sum(e);
    m = block_sum(m);
    if (threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_E), (unsigned long long)e);
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_M), (unsigned long long)m);
        __threadfence();
        if (atomicAdd(&ctl->up_blocks, 1u) == gridDim.x - 1) {
            __threadfence();
            ctl->E = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_E), 0ull);
            ctl->M = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_M), 0ull);
            ctl->up_blocks = 0;
        }
    }
}

// Bit-packed download: one warp ballot per 32 consecutive sites.
__global__ void k_to_bits(uint32_t *bits, const uint8_t *spins, uint32_t N) {
    const uint32_t words = (N + 31u) / 32u;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < words; w += warps) {
        const uint32_t i = w * 32u + lane;
        const uint32_t b = __ballot_sync(0xffffffffu, i < N && (spins[i] & 1u));
        if (lane == 0) bits[w] = b;
    }
}

cudaError_t launch_from_bits_measure(int dim, uint8_t *spins, const uint32_t *bits, Geometry g,
                                     DevCtl *ctl, cudaStream_t s) {
    if (g.L % 32 == 0) {
        if (dim == 2)
            k_from_bits_words<2><<<word_blocks(g), 256, 0, s>>>(spins, bits, g, ctl);
        else
            k_from_bits_words<3><<<word_blocks(g), 256, 0, s>>>(spins, bits, g, ctl);
        return cudaGetLastError();
    }
    const unsigned blocks = (unsigned)grid_for(g.N / g.L, 8192ull);
    const unsigned threads = g.L >= 256 ? 256 : 64;
    if (dim == 2)
        k_from_bits_measure<2><<<blocks, threads, 0, s>>>(spins, bits, g, ctl);
    else
        k_from_bits_measure<3><<<blocks, threads, 0, s>>>(spins, bits, g, ctl);
    return cudaGetLastError();
}

cudaError_t launch_to_bits(uint32_t *bits, const uint8_t *spins, uint32_t N, cudaStream_t s) {
    const unsigned long long words = (N + 31ull) / 32ull;
    k_to_bits<<<grid_for((words * 32ull + 255ull) / 256ull, 4096ull), 256, 0, s>>>(bits, spins, N);
    return cudaGetLastError();
}

// Expects a control block reset by k_reset_ctl (full sums and block count 0).
cudaError_t launch_from_pm1_measure(int dim, uint8_t *spins, const int8_t *src, Geometry g,
                                    DevCtl *ctl, cudaStream_t s) {
    const unsigned blocks = (unsigned)grid_for(g.N / g.L, 8192ull);
    const unsigned threads = g.L >= 256 ? 256 : 64;
    if (dim == 2)
        k_from_pm1_measure<2><<<blocks, threads, 0, s>>>(spins, src, g, ctl);
    else
        k_from_pm1_measure<3><<<blocks, threads, 0, s>>>(spins, src, g, ctl);
    return cudaGetLastError();
}

cudaError_t launch_from_pm1(uint8_t *spins, const int8_t *src, uint32_t N, DevCtl *ctl,
                            cudaStream_t s) {
    const unsigned blocks = grid_for((N + 255) / 256, 4096ull);
    k_from_pm1<<<blocks, 256, 0, s>>>(spins, src, N, ctl);
    return cudaGetLastError();
}

cudaError_t launch_to_pm1(int8_t *dst, const uint8_t *spins, uint32_t N, cudaStream_t s) {
    const unsigned blocks = grid_for((N + 255) / 256, 4096ull);
    k_to_pm1<<<blocks, 256, 0, s>>>(dst, spins, N);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void k_philox(uint32_t k0, uint32_t k1, const uint32_t *ctr, uint32_t *out,
                         unsigned long long n) {
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         k < n; k += (unsigned long long)gridDim.x * blockDim.x) {
        const Philox4 r = philox4x32_10(ctr[4 * k], ctr[4 * k + 1], ctr[4 * k + 2],
                                        ctr[4 * k + 3], k0, k1);
        out[4 * k] = r.v[0];
        out[4 * k + 1] = r.v[1];
        out[4 * k + 2] = r.v[2];
        out[4 * k + 3] = r.v[3];
    }
}

cudaError_t launch_philox(uint32_t k0, uint32_t k1, const uint32_t *ctr, uint32_t *out,
                          unsigned long long n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned blocks = grid_for((n + 255) / 256, 1024ull);
    k_philox<<<blocks, 256, 0, s>>>(k0, k1, ctr, out, n);
    return cudaGetLastError();
}

__global__ void k_reset_ctl(DevCtl *ctl, unsigned long long t) {
    ctl->t = t;
    ctl->last_C = 0;
    ctl->last_levels = 0;
    ctl->total_C = 0;
    ctl->status = 0;
    ctl->err_detail = 0;
    ctl->full_E = ctl->full_M = ctl->full_My = 0;
    ctl->up_blocks = 0;
    for (int k = 0; k < 4; ++k) ctl->cnt[k] = 0;
    ctl->dE = 0;
    ctl->bar_word = 0;
    ctl->bar_pub = 0;
    ctl->lo = ctl->hi = ctl->levels = ctl->done = 0;
    ctl->sig0bit = 0;
    ctl->t_end = t;
    ctl->rec_t0 = t;
    ctl->records = nullptr;
    ctl->cmd_seq = 0;
    ctl->st_updates = ctl->st_levels_local = ctl->st_levels_grid = 0;
    ctl->st_ns_local = ctl->st_ns_grid = ctl->st_ns_finish = 0;
    ctl->st_handoffs = ctl->st_grid_finishes = 0;
    ctl->st_start_ns = ctl->st_end_ns = 0;
    ctl->st_burst_updates = 0;
    ctl->st_bursts = 0;
    for (int k = 0; k < 4; ++k) ctl->st_ns_win[k] = 0;
    ctl->st_win_levels = 0;
    ctl->st_pregrown = 0;
    ctl->st_ns_win_first = ctl->st_win_regrown = ctl->st_win_fresh_grown = 0;
    for (int k = 0; k < 2; ++k)
        ctl->pg_next[k] = ctl->pg_stop[k] = ctl->pg_commit[k] = ctl->pg_done[k] = 0;
}

// Before every persistent launch: command sequence, barrier word and
// generation start from zero, so no CTA has to read them at start-up.
__global__ void k_prelaunch(DevCtl *ctl) {
    ctl->cmd_seq = 0;
    ctl->bar_word = 0;
    ctl->bar_pub = 0;
    ctl->dE = 0;
}

cudaError_t launch_prelaunch(DevCtl *ctl, cudaStream_t s) {
    k_prelaunch<<<1, 1, 0, s>>>(ctl);
    return cudaGetLastError();
}

cudaError_t launch_reset_ctl(DevCtl *ctl, unsigned long long t, cudaStream_t s) {
    k_reset_ctl<<<1, 1, 0, s>>>(ctl, t);
    return cudaGetLastError();
}

// Failure-detection self test: one CTA waits at a grid barrier that expects
// two, so only the time limit can end the wait.
__global__ void k_selftest_wait(DevCtl *scratch, unsigned long long wait_ns) {
    unsigned int gen = 0, phase = 0;
    team_barrier(scratch, 2u, gen, phase, true, wait_ns, 0x7E57u, nullptr);
}

cudaError_t launch_selftest_wait(DevCtl *scratch, unsigned long long wait_ns, cudaStream_t s) {
    k_selftest_wait<<<1, 32, 0, s>>>(scratch, wait_ns);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shared pieces of both schedules.

// Expands list[lo, hi) with all warps of the grid; new members go to
// list[hi + ...] through `counter`.
template <int DIM, typename Counter>
__device__ __forceinline__ void expand_range(const StepParams &p, uint32_t lo, uint32_t hi,
                                             uint32_t sig0bit, uint32_t tlo, uint32_t thi,
                                             Counter *counter) {
    const uint32_t warps_per_block = blockDim.x >> 5;
    const uint32_t gwarp = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
    const uint32_t nwarps = gridDim.x * warps_per_block;
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t base = lo + gwarp * 32u; base < hi; base += nwarps * 32u) {
        const uint32_t k = base + lane;
        Neighbours<DIM> nb;
        uint32_t won = 0;
        if (k < hi) won = expand_site<DIM>(p, __ldcg(p.list + k), sig0bit, tlo, thi, nb);
        uint32_t pos = hi + warp_reserve(counter, __popc(won));
#pragma unroll
        for (int s = 0; s < 2 * DIM; ++s) {
            if (won & (1u << s)) {
                if (pos < p.g.N) p.list[pos] = nb.packed[s];
                else raise_status(p.ctl, WOLFF_EINVAL, 0xC0FFu);
                ++pos;
            }
        }
    }
}

// Boundary-bond sum over list[0, C) for this CTA's share (grid-stride).
template <int DIM>
__device__ __forceinline__ long long boundary_range(const StepParams &p, uint32_t C,
                                                    uint32_t sig0bit) {
    long long acc = 0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < C;
         k += gridDim.x * blockDim.x) {
        uint32_t i;
        acc += boundary_term<DIM>(p, __ldcg(p.list + k), sig0bit, &i);
    }
    return acc;
}

// Unmark list[0, C) (grid-stride) and give the slots back their empty value.
template <int DIM>
__device__ __forceinline__ void unmark_range(const StepParams &p, uint32_t C, uint32_t sig0bit) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < C;
         k += gridDim.x * blockDim.x) {
        uint32_t c[DIM];
        unpack<DIM>(__ldcg(p.list + k), c);
        unmark_site(p.spins, site_index<DIM>(p.g, c), sig0bit);
        p.list[k] = kEmptySlot;
    }
}

// Closes update t: E, M, record, counters.  One thread.
__device__ __forceinline__ void finish_update(const StepParams &p, DevCtl *ctl,
                                              wolff_record *records, unsigned long long rec_index,
                                              uint32_t C, uint32_t levels, uint32_t sig0bit,
                                              unsigned long long t, long long dE_local) {
    const long long dE = *reinterpret_cast<volatile long long *>(&ctl->dE) + dE_local;
    const long long E = ctl->E + 2 * dE;
    const long long M = ctl->M + (sig0bit ? -2LL : 2LL) * (long long)C;
    ctl->E = E;
    ctl->M = M;
    ctl->dE = 0;
    ctl->cnt[0] = ctl->cnt[1] = ctl->cnt[2] = 0;
    ctl->last_C = C;
    ctl->last_levels = levels;
    ctl->total_C += C;
    ctl->t = t + 1;
    if (records) {
        wolff_record r;
        r.C = C;
        r.levels = levels;
        r.E_bond = E;
        r.M = M;
        records[rec_index] = r;
    }
}

// ---------------------------------------------------------------------------
// Persistent cooperative schedule: a leader CTA and worker CTAs.
//
// CTA 0 (the leader) runs every update.  While the wave front is small it
// grows the cluster alone -- frontier and cluster-list prefix in shared
// memory, __syncthreads as the level barrier -- which is the on-GPU form of
// the paper's hybrid (section 6: small wave fronts are cheaper on one
// processor).  When a level produces more than t_up new sites it publishes a
// GROW command and all CTAs expand the following levels together, separated
// by the relaxed team barrier, until a level produces t_down sites or fewer;
// then the workers go back to waiting and the leader continues alone.  A
// cluster that fits the shared-memory list and never went to the grid is
// closed by the leader alone; otherwise a FINISH command runs the energy and
// unmark passes on all CTAs, closed by full barriers.  t_up = 0 gives the
// plain grid-synchronous schedule (every level on all CTAs).  The leader
// keeps the chain state (t, E, M) in registers and writes it back at exit.

enum : unsigned int { kCmdGrow = 1, kCmdFinish = 2, kCmdExit = 3 };

struct SharedLocal {
    uint32_t front[2][kLocalFrontierCap];
    uint32_t list[kLocalListCap];
    unsigned int cnt[3];
    unsigned int sig0bit;
    unsigned int flag;
    unsigned int cmd[8];
};

// All CTAs: from the wave front list[lo, hi) (phase just published, entries
// appended at base + the barrier word's count), expand level after level until
// the next front is empty (*finished = true) or has t_down sites or fewer.
template <int DIM>
__device__ __forceinline__ bool grid_levels(const StepParams &p, unsigned int &gen,
                                            unsigned int &phase, uint32_t &lo, uint32_t &hi,
                                            uint32_t &level, uint32_t sig0bit, uint32_t tlo,
                                            uint32_t thi, bool *finished) {
    DevCtl *ctl = p.ctl;
    const uint32_t base = hi;
    const uint32_t warps_per_block = blockDim.x >> 5;
    const uint32_t gwarp = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
    const uint32_t nwarps = gridDim.x * warps_per_block;
    const uint32_t lane = threadIdx.x & 31;
    while (true) {
        for (uint32_t b = lo + gwarp * 32u; b < hi; b += nwarps * 32u) {
            const uint32_t k = b + lane;
            Neighbours<DIM> nb;
            uint32_t won = 0;
            if (k < hi) {
                const uint32_t packed = wait_slot(p, k);
                if (packed != kEmptySlot) won = expand_site<DIM>(p, packed, sig0bit, tlo, thi, nb);
            }
            uint32_t pos = base + warp_reserve(&ctl->bar_word, __popc(won));
#pragma unroll
            for (int s = 0; s < 2 * DIM; ++s) {
                if (won & (1u << s)) {
                    if (pos < p.g.N) p.list[pos] = nb.packed[s];
                    else raise_status(ctl, WOLFF_EINVAL, 0xC0FFu);
                    ++pos;
                }
            }
        }
        unsigned int total = 0;
        if (!team_barrier(ctl, gridDim.x, gen, phase, false, p.wait_ns, 1, &total)) return false;
        ++level;
        const uint32_t next_hi = base + total;
        if (next_hi < hi || next_hi > p.g.N) {   // cannot happen: each site joins once
            if (blockIdx.x == 0 && threadIdx.x == 0) raise_status(ctl, WOLFF_EINVAL, 0xC1u);
            return false;
        }
        const uint32_t added = next_hi - hi;
        lo = hi;
        hi = next_hi;
        if (added == 0) { *finished = true; return true; }
        if (added <= p.t_down) { *finished = false; return true; }
    }
}

// All CTAs: energy change over list[0, C), then unmark; closed by full
// barriers so that the unmark and the emptied slots are visible before the
// next update.  Returns the update's boundary sum in thread 0 of CTA 0.
template <int DIM>
__device__ __forceinline__ bool grid_finish(const StepParams &p, unsigned int &gen,
                                            unsigned int &phase, uint32_t C, uint32_t sig0bit,
                                            long long *dE_out) {
    DevCtl *ctl = p.ctl;
    long long acc = 0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < C;
         k += gridDim.x * blockDim.x) {
        const uint32_t packed = wait_slot(p, k);
        uint32_t i;
        if (packed != kEmptySlot) acc += boundary_term<DIM>(p, packed, sig0bit, &i);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0 && acc != 0)
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->dE), (unsigned long long)acc);
    if (!team_barrier(ctl, gridDim.x, gen, phase, true, p.wait_ns, 2, nullptr)) return false;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *dE_out = *reinterpret_cast<volatile long long *>(&ctl->dE);
    }
    unmark_range<DIM>(p, C, sig0bit);
    if (!team_barrier(ctl, gridDim.x, gen, phase, true, p.wait_ns, 3, nullptr)) return false;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->dE = 0;   // read above, before the barrier
    return true;
}

// Leader thread 0: start a new team phase (barrier word cleared while every
// worker is idle) and publish a command (release on cmd_seq).
__device__ __forceinline__ void publish(DevCtl *ctl, unsigned int &seq, unsigned int kind,
                                        uint32_t lo, uint32_t hi, uint32_t level,
                                        uint32_t sig0bit, unsigned long long t) {
    ctl->bar_word = 0;
    ctl->cmd_kind = kind;
    ctl->cmd_lo = lo;
    ctl->cmd_hi = hi;
    ctl->cmd_level = level;
    ctl->cmd_sig0bit = sig0bit;
    ctl->cmd_t = t;
    __threadfence();
    seq += 1;
    st_release_u32(&ctl->cmd_seq, seq);
}

template <int DIM>
__device__ void worker_loop(const StepParams &p, SharedLocal &sh, unsigned int &gen) {
    DevCtl *ctl = p.ctl;
    unsigned int seq = 0;
    while (true) {
        if (threadIdx.x == 0) {
            bool ok = true;
            const unsigned int v = bounded_wait_change(ctl, &ctl->cmd_seq, seq, &ctl->t,
                                                       p.wait_ns, 4, &ok);
            if (!ok) {
                sh.cmd[0] = kCmdExit;
            } else {
                seq = v;
                sh.cmd[0] = ld_volatile_u32(&ctl->cmd_kind);
                sh.cmd[1] = ctl->cmd_lo;
                sh.cmd[2] = ctl->cmd_hi;
                sh.cmd[3] = ctl->cmd_level;
                sh.cmd[4] = ctl->cmd_sig0bit;
                const unsigned long long t = ctl->cmd_t;
                sh.cmd[5] = (uint32_t)t;
                sh.cmd[6] = (uint32_t)(t >> 32);
            }
        }
        __syncthreads();
        const unsigned int kind = sh.cmd[0];
        uint32_t lo = sh.cmd[1], hi = sh.cmd[2], level = sh.cmd[3];
        const uint32_t sig0bit = sh.cmd[4], tlo = sh.cmd[5], thi = sh.cmd[6];
        __syncthreads();
        unsigned int phase = 0;
        if (kind == kCmdGrow) {
            bool finished = false;
            if (!grid_levels<DIM>(p, gen, phase, lo, hi, level, sig0bit, tlo, thi, &finished))
                return;
        } else if (kind == kCmdFinish) {
            long long dE = 0;
            if (!grid_finish<DIM>(p, gen, phase, hi, sig0bit, &dE)) return;
        } else {
            return;
        }
    }
}

template <int DIM>
__global__ void __launch_bounds__(512, 1) k_persistent(StepParams p) {
    DevCtl *ctl = p.ctl;
    __shared__ SharedLocal sh;
    unsigned int gen = 0;   // the pre-launch kernel zeroed the generation
    if (blockIdx.x != 0) {
        worker_loop<DIM>(p, sh, gen);
        return;
    }
    const bool t0 = threadIdx.x == 0;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t t_up = min(p.t_up, kLocalFrontierCap);
    unsigned int seq = 0;
    // chain state, kept by thread 0 in registers
    long long E = 0, M = 0;
    unsigned long long total_C = 0;
    uint32_t last_C = 0, last_levels = 0;
    unsigned long long st_local = 0, st_grid = 0, ns_local = 0, ns_grid = 0, ns_finish = 0;
    unsigned long long handoffs = 0, grid_fin = 0;
    if (t0) {
        ctl->st_start_ns = global_ns();
        E = ctl->E;
        M = ctl->M;
        total_C = ctl->total_C;
        last_C = ctl->last_C;
        last_levels = ctl->last_levels;
    }
    unsigned long long done = 0;
    for (unsigned long long u = 0; u < p.n; ++u) {
        const unsigned long long t = p.t0 + u;
        const uint32_t tlo = (uint32_t)t, thi = (uint32_t)(t >> 32);
        unsigned long long clk = 0;
        if (t0) {
            // a status latched before this launch (an invalid input lattice)
            // or during it stops the chain before the next seed is claimed,
            // so the lattice is left as the last completed update made it
            sh.flag = (u == 0 || (u & 31u) == 31u) ? ld_volatile_u32(&ctl->status) : 0u;
            if (sh.flag == 0u) {
                // seed: one uncontended XOR flips its bit 0 and returns its spin
                const uint32_t i0 = seed_site(p, t);
                unsigned int *w = reinterpret_cast<unsigned int *>(p.spins) + (i0 >> 2);
                const unsigned int sh0 = (i0 & 3u) * 8u;
                const uint32_t s0 = (atomicXor(w, 1u << sh0) >> sh0) & 1u;
                const uint32_t p0 = pack_index<DIM>(p.g, i0);
                p.list[0] = p0;
                sh.list[0] = p0;
                sh.front[0][0] = p0;
                sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
                sh.sig0bit = s0;
            }
            clk = global_ns();
        }
        __syncthreads();
        if (sh.flag != 0u) break;
        const uint32_t sig0bit = sh.sig0bit;
        uint32_t C = 1, f = 1, level = 0, cur = 0;
        bool went_grid = false;
        while (f > 0) {
            if (f > t_up) {
                // hand the wave front list[C-f, C) to all CTAs
                went_grid = true;
                unsigned long long g0 = 0;
                if (t0) {
                    g0 = global_ns();
                    ns_local += g0 - clk;
                    ++handoffs;
                    publish(ctl, seq, kCmdGrow, C - f, C, level, sig0bit, t);
                }
                __syncthreads();
                uint32_t lo = C - f, hi = C, phase = 0, lv0 = level;
                bool finished = false;
                if (!grid_levels<DIM>(p, gen, phase, lo, hi, level, sig0bit, tlo, thi,
                                      &finished))
                    return;
                C = hi;
                f = finished ? 0u : hi - lo;
                if (f) {   // back to the leader: load the small front
                    for (uint32_t k = threadIdx.x; k < f; k += blockDim.x)
                        sh.front[cur][k] = wait_slot(p, lo + k);
                    if (t0) sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
                }
                if (t0) {
                    st_grid += level - lv0;
                    clk = global_ns();
                    ns_grid += clk - g0;
                }
                __syncthreads();
                continue;
            }
            // one level on the leader alone
            const uint32_t nxt = cur ^ 1u;
            unsigned int *cnt = &sh.cnt[level % 3];
            if (t0) sh.cnt[(level + 1) % 3] = 0;
            for (uint32_t b = warp * 32u; b < f; b += nwarps * 32u) {
                const uint32_t k = b + lane;
                Neighbours<DIM> nb;
                uint32_t won = 0;
                if (k < f) won = expand_site<DIM>(p, sh.front[cur][k], sig0bit, tlo, thi, nb);
                uint32_t pos = warp_reserve(cnt, __popc(won));
#pragma unroll
                for (int s = 0; s < 2 * DIM; ++s) {
                    if (won & (1u << s)) {
                        const uint32_t gpos = C + pos;
                        if (gpos < p.g.N) p.list[gpos] = nb.packed[s];
                        else raise_status(ctl, WOLFF_EINVAL, 0xC3u);
                        if (gpos < kLocalListCap) sh.list[gpos] = nb.packed[s];
                        if (pos < kLocalFrontierCap) sh.front[nxt][pos] = nb.packed[s];
                        ++pos;
                    }
                }
            }
            __syncthreads();
            const uint32_t added = *cnt;
            ++level;
            if (t0) ++st_local;
            C += added;
            f = added;
            cur = nxt;
        }
        long long dE = 0;
        unsigned long long f0 = 0;
        if (t0) {
            f0 = global_ns();
            ns_local += f0 - clk;
        }
        if (went_grid || C > kLocalListCap) {
            if (t0) {
                ++grid_fin;
                publish(ctl, seq, kCmdFinish, 0, C, level, sig0bit, t);
            }
            __syncthreads();
            uint32_t phase = 0;
            if (!grid_finish<DIM>(p, gen, phase, C, sig0bit, &dE)) return;
        } else {
            // the leader closes a small cluster alone from its shared list
            long long acc = 0;
            for (uint32_t k = threadIdx.x; k < C; k += blockDim.x) {
                uint32_t i;
                acc += boundary_term<DIM>(p, sh.list[k], sig0bit, &i);
            }
            dE = block_sum(acc);
            __syncthreads();
            for (uint32_t k = threadIdx.x; k < C; k += blockDim.x) {
                uint32_t c[DIM];
                unpack<DIM>(sh.list[k], c);
                unmark_site(p.spins, site_index<DIM>(p.g, c), sig0bit);
                p.list[k] = kEmptySlot;
            }
        }
        if (t0) {
            E += 2 * dE;
            M += (sig0bit ? -2LL : 2LL) * (long long)C;
            total_C += C;
            last_C = C;
            last_levels = level;
            if (p.records) {
                wolff_record r;
                r.C = C;
                r.levels = level;
                r.E_bond = E;
                r.M = M;
                p.records[u] = r;
            }
            *reinterpret_cast<volatile unsigned long long *>(&ctl->t) = t + 1;   // progress
            ns_finish += global_ns() - f0;
        }
        ++done;
        __syncthreads();
    }
    if (t0) {
        ctl->E = E;
        ctl->M = M;
        ctl->total_C = total_C;
        ctl->last_C = last_C;
        ctl->last_levels = last_levels;
        ctl->t = p.t0 + done;
        ctl->st_updates += done;
        ctl->st_levels_local += st_local;
        ctl->st_levels_grid += st_grid;
        ctl->st_ns_local += ns_local;
        ctl->st_ns_grid += ns_grid;
        ctl->st_ns_finish += ns_finish;
        ctl->st_handoffs += handoffs;
        ctl->st_grid_finishes += grid_fin;
        ctl->st_end_ns = global_ns();
        publish(ctl, seq, kCmdExit, 0, 0, 0, 0, 0);
    }
}

const void *persistent_kernel(int dim) {
    return dim == 2 ? reinterpret_cast<const void *>(&k_persistent<2>)
                    : reinterpret_cast<const void *>(&k_persistent<3>);
}

int persistent_max_blocks_per_sm(int dim, int threads, int *err) {
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, persistent_kernel(dim), threads, 0);
    if (err) *err = (int)e;
    return n;
}

// ---------------------------------------------------------------------------
// Graph schedule: per-level kernels inside nested conditional WHILE nodes.

template <int DIM>
__global__ void k_graph_begin(StepParams p, cudaGraphConditionalHandle h_level) {
    DevCtl *ctl = p.ctl;
    const unsigned long long t = ctl->t;
    const uint32_t i0 = seed_site(p, t);
    const uint32_t sig0bit = (p.spins[i0] >> 1) & 1u;
    claim_site(p.spins, i0, sig0bit);
    p.list[0] = pack_index<DIM>(p.g, i0);
    ctl->sig0bit = sig0bit;
    ctl->lo = 0;
    ctl->hi = 1;
    ctl->levels = 0;
    ctl->cnt[0] = 0;
    ctl->done = 0;
    ctl->dE = 0;
    cudaGraphSetConditional(h_level, 1u);
}

// Last-CTA-done epilogue: the CTA that finishes last publishes the next
// frontier and decides whether the WHILE loop continues.
__device__ __forceinline__ bool last_block_done(DevCtl *ctl) {
    __shared__ unsigned int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(&ctl->done, 1u) == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0u;
}

template <int DIM>
__global__ void __launch_bounds__(1024) k_graph_level(StepParams p,
                                                      cudaGraphConditionalHandle h_level) {
    DevCtl *ctl = p.ctl;
    const unsigned long long t = ctl->t;
    const uint32_t lo = ctl->lo, hi = ctl->hi, sig0bit = ctl->sig0bit;
    expand_range<DIM>(p, lo, hi, sig0bit, (uint32_t)t, (uint32_t)(t >> 32), &ctl->cnt[0]);
    if (last_block_done(ctl) && threadIdx.x == 0) {
        uint32_t added = ld_volatile_u32(&ctl->cnt[0]);
        if (added > p.g.N - hi) {   // cannot happen: each site joins once
            raise_status(ctl, WOLFF_EINVAL, 0xC2u);
            added = 0;
        }
        ctl->cnt[0] = 0;
        ctl->done = 0;
        ctl->levels += 1;
        ctl->lo = hi;
        ctl->hi = hi + added;
        cudaGraphSetConditional(h_level, added != 0u ? 1u : 0u);
    }
}

template <int DIM>
__global__ void __launch_bounds__(1024) k_graph_boundary(StepParams p) {
    DevCtl *ctl = p.ctl;
    const long long acc = block_sum(boundary_range<DIM>(p, ctl->hi, ctl->sig0bit));
    if (threadIdx.x == 0 && acc != 0)
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->dE), (unsigned long long)acc);
}

template <int DIM>
__global__ void __launch_bounds__(1024) k_graph_finish(StepParams p,
                                                       cudaGraphConditionalHandle h_update) {
    DevCtl *ctl = p.ctl;
    const uint32_t C = ctl->hi, sig0bit = ctl->sig0bit;
    unmark_range<DIM>(p, C, sig0bit);
    if (last_block_done(ctl) && threadIdx.x == 0) {
        const unsigned long long t = ctl->t;
        ctl->done = 0;
        finish_update(p, ctl, ctl->records, t - ctl->rec_t0, C, ctl->levels, sig0bit, t, 0);
        cudaGraphSetConditional(h_update, (t + 1 < ctl->t_end) ? 1u : 0u);
    }
}

__global__ void k_graph_call(DevCtl *ctl, unsigned long long n, wolff_record *records) {
    ctl->t_end = ctl->t + n;
    ctl->rec_t0 = ctl->t;
    ctl->records = records;
}

cudaError_t launch_graph_call(DevCtl *ctl, unsigned long long n, wolff_record *records,
                              cudaStream_t s) {
    k_graph_call<<<1, 1, 0, s>>>(ctl, n, records);
    return cudaGetLastError();
}

static cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t *node, const cudaGraphNode_t *dep,
                              size_t ndep, const void *fn, unsigned blocks, unsigned threads,
                              void **args) {
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeKernel;
    np.kernel.func = const_cast<void *>(fn);
    np.kernel.gridDim = dim3(blocks);
    np.kernel.blockDim = dim3(threads);
    np.kernel.sharedMemBytes = 0;
    np.kernel.kernelParams = args;
    return cudaGraphAddNode(node, g, dep, nullptr, ndep, &np);
}

template <int DIM>
static cudaError_t build_graph_dim(const StepParams &p_in, int blocks, int threads,
                                   cudaGraphExec_t *exec, cudaGraph_t *out_graph) {
    cudaError_t e;
    cudaGraph_t g = nullptr;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
    StepParams p = p_in;
    cudaGraphConditionalHandle h_update, h_level;
    if ((e = cudaGraphConditionalHandleCreate(&h_update, g, 1, cudaGraphCondAssignDefault)) !=
        cudaSuccess)
        goto fail;
    {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h_update;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t outer;
        if ((e = cudaGraphAddNode(&outer, g, nullptr, nullptr, 0, &cp)) != cudaSuccess) goto fail;
        cudaGraph_t body = cp.conditional.phGraph_out[0];

        if ((e = cudaGraphConditionalHandleCreate(&h_level, body, 0, 0)) != cudaSuccess) goto fail;
        cudaGraphNode_t n_begin, n_loop, n_boundary, n_finish;
        void *args_begin[] = {&p, &h_level};
        if ((e = add_kernel(body, &n_begin, nullptr, 0,
                            reinterpret_cast<const void *>(&k_graph_begin<DIM>), 1, 1,
                            args_begin)) != cudaSuccess)
            goto fail;
        cudaGraphNodeParams lp = {};
        lp.type = cudaGraphNodeTypeConditional;
        lp.conditional.handle = h_level;
        lp.conditional.type = cudaGraphCondTypeWhile;
        lp.conditional.size = 1;
        if ((e = cudaGraphAddNode(&n_loop, body, &n_begin, nullptr, 1, &lp)) != cudaSuccess)
            goto fail;
        cudaGraph_t level_body = lp.conditional.phGraph_out[0];
        cudaGraphNode_t n_level;
        void *args_level[] = {&p, &h_level};
        if ((e = add_kernel(level_body, &n_level, nullptr, 0,
                            reinterpret_cast<const void *>(&k_graph_level<DIM>), blocks, threads,
                            args_level)) != cudaSuccess)
            goto fail;
        void *args_boundary[] = {&p};
        if ((e = add_kernel(body, &n_boundary, &n_loop, 1,
                            reinterpret_cast<const void *>(&k_graph_boundary<DIM>), blocks,
                            threads, args_boundary)) != cudaSuccess)
            goto fail;
        void *args_finish[] = {&p, &h_update};
        if ((e = add_kernel(body, &n_finish, &n_boundary, 1,
                            reinterpret_cast<const void *>(&k_graph_finish<DIM>), blocks, threads,
                            args_finish)) != cudaSuccess)
            goto fail;
    }
    if ((e = cudaGraphInstantiate(exec, g, 0)) != cudaSuccess) goto fail;
    *out_graph = g;
    return cudaSuccess;
fail:
    cudaGraphDestroy(g);
    return e;
}

cudaError_t build_update_graph(int dim, const StepParams &p, int blocks, int threads,
                               cudaGraphExec_t *exec, cudaGraph_t *graph) {
    return dim == 2 ? build_graph_dim<2>(p, blocks, threads, exec, graph)
                    : build_graph_dim<3>(p, blocks, threads, exec, graph);
}

}  // namespace wolff
