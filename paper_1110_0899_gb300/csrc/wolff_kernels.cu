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

__global__ void k_zero_full(DevCtl *ctl) {
    ctl->full_E = 0;
    ctl->full_M = 0;
}

__global__ void k_full_to_chain(DevCtl *ctl) {
    ctl->E = ctl->full_E;
    ctl->M = ctl->full_M;
}

cudaError_t launch_measure_full(int dim, const uint8_t *spins, Geometry g, DevCtl *ctl,
                                int set_chain, cudaStream_t s) {
    k_zero_full<<<1, 1, 0, s>>>(ctl);
    const uint32_t rows = g.N / g.L;
    const unsigned blocks = grid_for(rows, 8192ull);
    const unsigned threads = g.L >= 256 ? 256 : 64;
    if (dim == 2)
        k_measure_full<2><<<blocks, threads, 0, s>>>(spins, g, ctl);
    else
        k_measure_full<3><<<blocks, threads, 0, s>>>(spins, g, ctl);
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
    for (int k = 0; k < 4; ++k) ctl->cnt[k] = 0;
    ctl->dE = 0;
    ctl->bar_count = 0;
    ctl->bar_gen = 0;
    ctl->lo = ctl->hi = ctl->levels = ctl->done = 0;
    ctl->sig0bit = 0;
    ctl->t_end = t;
    ctl->rec_t0 = t;
    ctl->records = nullptr;
}

cudaError_t launch_reset_ctl(DevCtl *ctl, unsigned long long t, cudaStream_t s) {
    k_reset_ctl<<<1, 1, 0, s>>>(ctl, t);
    return cudaGetLastError();
}

// Failure-detection self test: one CTA waits at a grid barrier that expects
// two, so only the time limit can end the wait.
__global__ void k_selftest_wait(DevCtl *scratch, unsigned long long wait_ns) {
    unsigned int gen = 0;
    grid_barrier(scratch, 2u, gen, wait_ns, 0x7E57u);
}

cudaError_t launch_selftest_wait(DevCtl *scratch, unsigned long long wait_ns, cudaStream_t s) {
    k_selftest_wait<<<1, 32, 0, s>>>(scratch, wait_ns);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shared pieces of both schedules.

// Expands list[lo, hi) with all warps of the grid; new members go to
// list[hi + ...] through `counter`.
template <int DIM>
__device__ __forceinline__ void expand_range(const StepParams &p, uint32_t lo, uint32_t hi,
                                             uint32_t sig0bit, uint32_t tlo, uint32_t thi,
                                             unsigned int *counter) {
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

// Unmark: both bits of every member take the new spin (opposite of sigma0).
template <int DIM>
__device__ __forceinline__ void unmark_range(const StepParams &p, uint32_t C, uint32_t sig0bit) {
    const uint8_t v = sig0bit ? 0x00 : 0x03;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < C;
         k += gridDim.x * blockDim.x) {
        uint32_t c[DIM];
        unpack<DIM>(__ldcg(p.list + k), c);
        p.spins[site_index<DIM>(p.g, c)] = v;
    }
}

// Closes update t: E, M, record, counters.  One thread.
__device__ __forceinline__ void finish_update(const StepParams &p, DevCtl *ctl,
                                              wolff_record *records, unsigned long long rec_index,
                                              uint32_t C, uint32_t levels, uint32_t sig0bit,
                                              unsigned long long t) {
    const long long dE = *reinterpret_cast<volatile long long *>(&ctl->dE);
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
// Persistent cooperative schedule.
template <int DIM>
__global__ void __launch_bounds__(1024) k_persistent(StepParams p) {
    DevCtl *ctl = p.ctl;
    __shared__ unsigned int s_gen;
    if (threadIdx.x == 0) s_gen = ld_volatile_u32(&ctl->bar_gen);
    __syncthreads();
    unsigned int gen = s_gen;   // meaningful in thread 0 only
    const unsigned int nblocks = gridDim.x;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;

    for (unsigned long long u = 0; u < p.n; ++u) {
        const unsigned long long t = p.t0 + u;
        const uint32_t tlo = (uint32_t)t, thi = (uint32_t)(t >> 32);
        const uint32_t i0 = seed_site(p, t);
        // bit 1 holds the spin at the start of the update and never changes
        // during growth, so every CTA can read the seed spin at any time
        const uint32_t sig0bit = (__ldcg(p.spins + i0) >> 1) & 1u;
        if (leader) {
            claim_site(p.spins, i0, sig0bit);
            p.list[0] = pack_index<DIM>(p.g, i0);
        }
        uint32_t lo = 0, hi = 1, level = 0;
        while (true) {
            expand_range<DIM>(p, lo, hi, sig0bit, tlo, thi, &ctl->cnt[level % 3]);
            if (leader) ctl->cnt[(level + 1) % 3] = 0;
            if (!grid_barrier(ctl, nblocks, gen, p.wait_ns, 1)) return;
            const uint32_t added = ld_volatile_u32(&ctl->cnt[level % 3]);
            ++level;
            if (added == 0) break;
            if (added > p.g.N - hi) {   // cannot happen: each site joins once
                if (leader) raise_status(ctl, WOLFF_EINVAL, 0xC1u);
                return;
            }
            lo = hi;
            hi += added;
        }
        const uint32_t C = hi;
        const long long acc = block_sum(boundary_range<DIM>(p, C, sig0bit));
        if (threadIdx.x == 0 && acc != 0)
            atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->dE), (unsigned long long)acc);
        if (!grid_barrier(ctl, nblocks, gen, p.wait_ns, 2)) return;
        unmark_range<DIM>(p, C, sig0bit);
        if (leader) finish_update(p, ctl, p.records, u, C, level, sig0bit, t);
        if (!grid_barrier(ctl, nblocks, gen, p.wait_ns, 3)) return;
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
        finish_update(p, ctl, ctl->records, t - ctl->rec_t0, C, ctl->levels, sig0bit, t);
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
