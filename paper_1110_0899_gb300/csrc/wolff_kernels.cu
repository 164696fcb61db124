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
    grid_sync(scratch, 2u, gen, wait_ns, 0x7E57u, nullptr, nullptr);
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
// by the bounded grid barrier, until a level produces t_down sites or fewer;
// then the workers go back to waiting and the leader continues alone.  A
// cluster that fits the shared-memory list and never went to the grid is
// closed by the leader alone; otherwise a FINISH command runs the energy and
// unmark passes on all CTAs.  t_up = 0 gives the plain grid-synchronous
// schedule (every level on all CTAs).

enum : unsigned int { kCmdGrow = 1, kCmdFinish = 2, kCmdExit = 3 };

struct SharedLocal {
    uint32_t front[2][kLocalFrontierCap];
    uint32_t list[kLocalListCap];
    unsigned int cnt[3];
    unsigned int flag;
    unsigned int cmd[8];
};

// All CTAs: expand list[lo, hi) level after level until the next frontier is
// empty (*finished = true) or holds t_down sites or fewer.
template <int DIM>
__device__ __forceinline__ bool grid_levels(const StepParams &p, unsigned int &gen, uint32_t &lo,
                                            uint32_t &hi, uint32_t &level, uint32_t sig0bit,
                                            uint32_t tlo, uint32_t thi, bool *finished) {
    DevCtl *ctl = p.ctl;
    while (true) {
        expand_range<DIM>(p, lo, hi, sig0bit, tlo, thi, &ctl->cnt[0]);
        unsigned int added = 0;
        if (!grid_sync(ctl, gridDim.x, gen, p.wait_ns, 1, &ctl->cnt[0], &added)) return false;
        ++level;
        if (added > p.g.N - hi) {   // cannot happen: every site joins at most once
            if (blockIdx.x == 0 && threadIdx.x == 0) raise_status(ctl, WOLFF_EINVAL, 0xC1u);
            return false;
        }
        lo = hi;
        hi += added;
        if (added == 0) { *finished = true; return true; }
        if (added <= p.t_down) { *finished = false; return true; }
    }
}

// All CTAs: energy change over list[0, C), then unmark, then close the update.
template <int DIM>
__device__ __forceinline__ bool grid_finish(const StepParams &p, unsigned int &gen, uint32_t C,
                                            uint32_t levels, uint32_t sig0bit,
                                            unsigned long long t, unsigned long long rec) {
    DevCtl *ctl = p.ctl;
    const long long acc = block_sum(boundary_range<DIM>(p, C, sig0bit));
    if (threadIdx.x == 0 && acc != 0)
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->dE), (unsigned long long)acc);
    if (!grid_sync(ctl, gridDim.x, gen, p.wait_ns, 2, nullptr, nullptr)) return false;
    unmark_range<DIM>(p, C, sig0bit);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        finish_update(p, ctl, p.records, rec, C, levels, sig0bit, t, 0);
    return grid_sync(ctl, gridDim.x, gen, p.wait_ns, 3, nullptr, nullptr);
}

// Leader thread 0: publish a command to the workers (release on cmd_seq).
__device__ __forceinline__ void publish(DevCtl *ctl, unsigned int &seq, unsigned int kind,
                                        uint32_t lo, uint32_t hi, uint32_t level,
                                        uint32_t sig0bit, unsigned long long t,
                                        unsigned long long rec) {
    ctl->cmd_kind = kind;
    ctl->cmd_lo = lo;
    ctl->cmd_hi = hi;
    ctl->cmd_level = level;
    ctl->cmd_sig0bit = sig0bit;
    ctl->cmd_t = t;
    ctl->cmd_rec = rec;
    __threadfence();
    seq += 1;
    st_release_u32(&ctl->cmd_seq, seq);
}

template <int DIM>
__device__ void worker_loop(const StepParams &p, SharedLocal &sh, unsigned int &gen,
                            unsigned int seq) {
    DevCtl *ctl = p.ctl;
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
                const unsigned long long t = ctl->cmd_t, rec = ctl->cmd_rec;
                sh.cmd[5] = (uint32_t)t;
                sh.cmd[6] = (uint32_t)(t >> 32);
                sh.cmd[7] = (uint32_t)rec;
            }
        }
        __syncthreads();
        const unsigned int kind = sh.cmd[0];
        uint32_t lo = sh.cmd[1], hi = sh.cmd[2], level = sh.cmd[3];
        const uint32_t sig0bit = sh.cmd[4], tlo = sh.cmd[5], thi = sh.cmd[6];
        __syncthreads();
        if (kind == kCmdGrow) {
            bool finished = false;
            if (!grid_levels<DIM>(p, gen, lo, hi, level, sig0bit, tlo, thi, &finished)) return;
        } else if (kind == kCmdFinish) {
            const unsigned long long t = ((unsigned long long)thi << 32) | tlo;
            if (!grid_finish<DIM>(p, gen, hi, level, sig0bit, t, 0)) return;
        } else {
            return;
        }
    }
}

template <int DIM>
__global__ void __launch_bounds__(1024) k_persistent(StepParams p) {
    DevCtl *ctl = p.ctl;
    __shared__ SharedLocal sh;
    __shared__ unsigned int s_gen, s_seq;
    if (threadIdx.x == 0) {
        s_gen = ld_volatile_u32(&ctl->bar_gen);
        s_seq = ld_volatile_u32(&ctl->cmd_seq);
    }
    __syncthreads();
    unsigned int gen = s_gen;   // meaningful in thread 0
    unsigned int seq = s_seq;
    // every CTA has read the command sequence before the leader can publish
    if (!grid_sync(ctl, gridDim.x, gen, p.wait_ns, 5, nullptr, nullptr)) return;
    if (blockIdx.x != 0) {
        worker_loop<DIM>(p, sh, gen, seq);
        return;
    }
    const bool t0 = threadIdx.x == 0;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t t_up = min(p.t_up, kLocalFrontierCap);

    for (unsigned long long u = 0; u < p.n; ++u) {
        const unsigned long long t = p.t0 + u;
        const uint32_t tlo = (uint32_t)t, thi = (uint32_t)(t >> 32);
        const uint32_t i0 = seed_site(p, t);
        const uint32_t sig0bit = (p.spins[i0] >> 1) & 1u;
        if (t0) {
            claim_site(p.spins, i0, sig0bit);
            const uint32_t p0 = pack_index<DIM>(p.g, i0);
            p.list[0] = p0;
            sh.list[0] = p0;
            sh.front[0][0] = p0;
            sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
            sh.flag = ld_volatile_u32(&ctl->status);
        }
        __syncthreads();
        if (sh.flag != 0u) break;
        uint32_t C = 1, f = 1, level = 0, cur = 0;
        bool went_grid = false, ok = true;
        while (f > 0) {
            if (f > t_up) {
                // hand the wave front list[C-f, C) to all CTAs
                went_grid = true;
                if (t0) publish(ctl, seq, kCmdGrow, C - f, C, level, sig0bit, t, u);
                uint32_t lo = C - f, hi = C;
                bool finished = false;
                if (!grid_levels<DIM>(p, gen, lo, hi, level, sig0bit, tlo, thi, &finished)) {
                    ok = false;
                    break;
                }
                C = hi;
                f = finished ? 0u : hi - lo;
                if (f) {   // back to the leader: load the small front
                    for (uint32_t k = threadIdx.x; k < f; k += blockDim.x)
                        sh.front[cur][k] = __ldcg(p.list + lo + k);
                    if (t0) sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
                    __syncthreads();
                }
                continue;
            }
            // one level on the leader alone
            const uint32_t nxt = cur ^ 1u;
            unsigned int *cnt = &sh.cnt[level % 3];
            if (t0) sh.cnt[(level + 1) % 3] = 0;
            for (uint32_t base = warp * 32u; base < f; base += nwarps * 32u) {
                const uint32_t k = base + lane;
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
            C += added;
            f = added;
            cur = nxt;
        }
        if (!ok) return;
        if (went_grid || C > kLocalListCap) {
            if (t0) publish(ctl, seq, kCmdFinish, 0, C, level, sig0bit, t, u);
            if (!grid_finish<DIM>(p, gen, C, level, sig0bit, t, u)) return;
        } else {
            // the leader closes a small cluster alone from its shared list
            long long acc = 0;
            for (uint32_t k = threadIdx.x; k < C; k += blockDim.x) {
                uint32_t i;
                acc += boundary_term<DIM>(p, sh.list[k], sig0bit, &i);
            }
            acc = block_sum(acc);
            __syncthreads();
            const uint8_t v = sig0bit ? 0x00 : 0x03;
            for (uint32_t k = threadIdx.x; k < C; k += blockDim.x) {
                uint32_t c[DIM];
                unpack<DIM>(sh.list[k], c);
                p.spins[site_index<DIM>(p.g, c)] = v;
            }
            if (t0) finish_update(p, ctl, p.records, u, C, level, sig0bit, t, acc);
            __syncthreads();
        }
    }
    if (t0) publish(ctl, seq, kCmdExit, 0, 0, 0, 0, 0, 0);
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
