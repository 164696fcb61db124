// wolff_potts.cu -- the q-state Potts single-cluster update on a team.
//
// Section 6 of the paper names the Potts model as the straightforward
// extension of its GPU cluster growth.  H = -J sum_<ij> delta(c_i, c_j),
// colours 0..q-1 (q <= 64).  Update t: seed site from lane 0 of the seed
// draw, new colour c' = (c0 + 1 + floor(x1 (q-1) / 2^32)) mod q from lane 1;
// the cluster grows through bonds to neighbours of colour c0 active with
// p = 1 - exp(-J/T) (the same bond words as the Ising update); every member
// then takes c'.  With q = 2 the chain is the Ising chain of coupling J/2.
//
// Byte of a site: bits 0..5 colour, bit 7 "claimed in this update".  Colours
// do not change while a cluster grows, so a neighbour whose colour read c0 is
// claimable until someone sets its bit 7; the claim is one atomicOr of bit 7
// on the containing word (idempotent: exactly one claimer sees it clear).
// The flip XORs each member's byte from (c0 | 0x80) to c', which commutes
// with claims of neighbouring bytes in the same word.  Observables: the
// satisfied-bond count E_bond and N0 (sites of colour 0) in the M field.
//
// Schedule: one thread-block cluster per lattice as in wolff_team.cu -- the
// leader CTA grows small fronts alone, larger ones are shared by the team
// with distributed-shared-memory counters and the cluster barrier.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "wolff_device.cuh"

namespace cg = cooperative_groups;

namespace wolff {

namespace {

constexpr uint8_t kColourMask = 0x3F;
constexpr uint8_t kClaimBit = 0x80;

enum : unsigned int { kPottsLevels = 1, kPottsFinish = 2, kPottsExit = 3 };

struct PottsShared {
    uint32_t front[2][kLocalFrontierCap];
    uint32_t list[kLocalListCap];
    unsigned int cnt[3];
    unsigned int seed[3];   // c0, c', unused
    unsigned int cmd[8];    // kind, lo, hi, level, c0, c', t_lo, t_hi
    unsigned long long dE;  // team boundary sum (leader's copy)
};

// Claims every neighbour of colour c0 behind an active bond.  Returns the
// mask of neighbour slots won; nb receives their coordinates.
template <int DIM>
__device__ __forceinline__ uint32_t potts_expand(const StepParams &p, uint32_t packed,
                                                 uint32_t c0, uint32_t tlo, uint32_t thi,
                                                 Neighbours<DIM> &nb) {
    uint32_t i;
    neighbours<DIM>(p.g, packed, &i, nb);
    uint8_t v[2 * DIM];
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) v[s] = __ldcg(p.spins + nb.idx[s]);
    uint32_t owners[DIM + 1];
    owners[0] = i;
#pragma unroll
    for (int d = 0; d < DIM; ++d) owners[d + 1] = nb.idx[2 * d + 1];
    Philox4 draw[DIM + 1];
    philox4x32_10_lanes<DIM + 1>(owners, tlo, thi, kTagBond, p.key0, p.key1, draw);
    uint32_t want = 0;
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) {
        const int d = s >> 1;
        const uint32_t r = (s & 1) ? draw[d + 1].v[d] : draw[0].v[d];
        if ((v[s] & (kColourMask | kClaimBit)) == c0 && (unsigned long long)r < p.thr)
            want |= 1u << s;
    }
    unsigned int old[2 * DIM];
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) {
        old[s] = 0;
        if (want & (1u << s)) {
            unsigned int *w = reinterpret_cast<unsigned int *>(p.spins) + (nb.idx[s] >> 2);
            old[s] = atomicOr(w, (unsigned int)kClaimBit << ((nb.idx[s] & 3u) * 8u));
        }
    }
    uint32_t won = 0;
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) {
        const unsigned int bit = (unsigned int)kClaimBit << ((nb.idx[s] & 3u) * 8u);
        if ((want & (1u << s)) && (old[s] & bit) == 0u) won |= 1u << s;
    }
    return won;
}

// Energy change of one member: every neighbour outside the cluster turns a
// bond from delta(c0, c_j) to delta(c', c_j); bonds inside stay satisfied.
template <int DIM>
__device__ __forceinline__ int potts_boundary(const StepParams &p, uint32_t packed, uint32_t c0,
                                              uint32_t cn) {
    uint32_t i;
    Neighbours<DIM> nb;
    neighbours<DIM>(p.g, packed, &i, nb);
    int acc = 0;
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) {
        const uint32_t v = __ldcg(p.spins + nb.idx[s]);
        if (v & kClaimBit) continue;
        const uint32_t cj = v & kColourMask;
        acc += (int)(cj == cn) - (int)(cj == c0);
    }
    return acc;
}

__device__ __forceinline__ void potts_flip(uint8_t *spins, uint32_t j, uint32_t c0, uint32_t cn) {
    unsigned int *w = reinterpret_cast<unsigned int *>(spins) + (j >> 2);
    atomicXor(w, ((c0 | kClaimBit) ^ cn) << ((j & 3u) * 8u));
}

template <int DIM>
__device__ void potts_team_levels(const StepParams &p, PottsShared &sh, cg::cluster_group &cl,
                                  uint32_t &lo, uint32_t &hi, uint32_t &level, uint32_t c0,
                                  uint32_t tlo, uint32_t thi, bool *finished) {
    PottsShared *lead = cl.map_shared_rank(&sh, 0);
    const unsigned int rank = cl.block_rank(), cs = cl.num_blocks();
    const uint32_t warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t gw = rank * warps + warp, nw = cs * warps;
    while (true) {
        unsigned int *cnt = &lead->cnt[level % 3];
        if (rank == 0 && threadIdx.x == 0) sh.cnt[(level + 1) % 3] = 0;
        for (uint32_t b = lo + gw * 32u; b < hi; b += nw * 32u) {
            const uint32_t k = b + lane;
            Neighbours<DIM> nb;
            uint32_t won = 0;
            if (k < hi) won = potts_expand<DIM>(p, __ldcg(p.list + k), c0, tlo, thi, nb);
            uint32_t pos = hi + warp_reserve(cnt, __popc(won));
#pragma unroll
            for (int s = 0; s < 2 * DIM; ++s) {
                if (won & (1u << s)) {
                    if (pos < p.g.N) p.list[pos] = nb.packed[s];
                    else raise_status(p.ctl, WOLFF_EINVAL, 0xE0u);
                    ++pos;
                }
            }
        }
        cl.sync();
        uint32_t added = *reinterpret_cast<volatile unsigned int *>(cnt);
        ++level;
        if (added > p.g.N - hi) {
            if (rank == 0 && threadIdx.x == 0) raise_status(p.ctl, WOLFF_EINVAL, 0xE1u);
            added = 0;
        }
        lo = hi;
        hi += added;
        if (added == 0 || added <= p.t_down) {
            *finished = added == 0;
            cl.sync();   // every CTA has read the count before the leader reuses it
            return;
        }
    }
}

template <int DIM>
__device__ long long potts_team_finish(const StepParams &p, PottsShared &sh, cg::cluster_group &cl,
                                       uint32_t C, uint32_t c0, uint32_t cn) {
    PottsShared *lead = cl.map_shared_rank(&sh, 0);
    const unsigned int rank = cl.block_rank(), cs = cl.num_blocks();
    const uint32_t tid = rank * blockDim.x + threadIdx.x, nt = cs * blockDim.x;
    long long acc = 0;
    for (uint32_t k = tid; k < C; k += nt) acc += potts_boundary<DIM>(p, __ldcg(p.list + k), c0, cn);
    acc = block_sum(acc);
    if (threadIdx.x == 0 && acc != 0) atomicAdd(&lead->dE, (unsigned long long)acc);
    cl.sync();
    long long dE = 0;
    if (rank == 0 && threadIdx.x == 0) {
        dE = (long long)sh.dE;
        sh.dE = 0;
    }
    for (uint32_t k = tid; k < C; k += nt) {
        uint32_t c[DIM];
        unpack<DIM>(__ldcg(p.list + k), c);
        potts_flip(p.spins, site_index<DIM>(p.g, c), c0, cn);
        p.list[k] = kEmptySlot;
    }
    cl.sync();
    return dE;
}

template <int DIM>
__device__ void potts_worker(const StepParams &p, PottsShared &sh, cg::cluster_group &cl) {
    PottsShared *lead = cl.map_shared_rank(&sh, 0);
    while (true) {
        cl.sync();
        const volatile unsigned int *cmd = lead->cmd;
        const unsigned int kind = cmd[0];
        uint32_t lo = cmd[1], hi = cmd[2], level = cmd[3];
        const uint32_t c0 = cmd[4], cn = cmd[5], tlo = cmd[6], thi = cmd[7];
        if (kind == kPottsLevels) {
            bool finished = false;
            potts_team_levels<DIM>(p, sh, cl, lo, hi, level, c0, tlo, thi, &finished);
        } else if (kind == kPottsFinish) {
            potts_team_finish<DIM>(p, sh, cl, hi, c0, cn);
        } else {
            cl.sync();   // the leader's shared memory outlives every remote read
            return;
        }
    }
}

__device__ __forceinline__ void potts_announce(PottsShared &sh, cg::cluster_group &cl,
                                               unsigned int kind, uint32_t lo, uint32_t hi,
                                               uint32_t level, uint32_t c0, uint32_t cn,
                                               unsigned long long t) {
    if (threadIdx.x == 0) {
        sh.cmd[0] = kind;
        sh.cmd[1] = lo;
        sh.cmd[2] = hi;
        sh.cmd[3] = level;
        sh.cmd[4] = c0;
        sh.cmd[5] = cn;
        sh.cmd[6] = (uint32_t)t;
        sh.cmd[7] = (uint32_t)(t >> 32);
        sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
    }
    cl.sync();
}

template <int DIM>
__device__ void potts_leader(const StepParams &p, PottsShared &sh, cg::cluster_group &cl) {
    DevCtl *ctl = p.ctl;
    const bool t0 = threadIdx.x == 0;
    const bool has_team = cl.num_blocks() > 1;
    const uint32_t nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t q = p.q;
    long long E = 0, N0 = 0;
    unsigned long long total_C = 0;
    uint32_t last_C = 0, last_levels = 0;
    if (t0) {
        ctl->st_start_ns = global_ns();
        E = ctl->E;
        N0 = ctl->M;
        total_C = ctl->total_C;
        last_C = ctl->last_C;
        last_levels = ctl->last_levels;
        sh.dE = 0;
    }
    for (unsigned long long u = 0; u < p.n; ++u) {
        const unsigned long long t = p.t0 + u;
        const uint32_t tlo = (uint32_t)t, thi = (uint32_t)(t >> 32);
        if (t0) {
            const Philox4 r = philox4x32_10(0u, tlo, thi, kTagSeed, p.key0, p.key1);
            const uint32_t i0 = (uint32_t)(((unsigned long long)r.v[0] * p.g.N) >> 32);
            unsigned int *w = reinterpret_cast<unsigned int *>(p.spins) + (i0 >> 2);
            const unsigned int sh0 = (i0 & 3u) * 8u;
            const uint32_t c0 = (atomicOr(w, (unsigned int)kClaimBit << sh0) >> sh0) & kColourMask;
            const uint32_t cn =
                (c0 + 1u + (uint32_t)(((unsigned long long)r.v[1] * (q - 1u)) >> 32)) % q;
            const uint32_t p0 = pack_index<DIM>(p.g, i0);
            p.list[0] = p0;
            sh.list[0] = p0;
            sh.front[0][0] = p0;
            sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
            sh.seed[0] = c0;
            sh.seed[1] = cn;
        }
        __syncthreads();
        const uint32_t c0 = sh.seed[0], cn = sh.seed[1];
        uint32_t C = 1, f = 1, level = 0, cur = 0;
        bool went_team = false;
        while (f > 0) {
            if (has_team && f > p.t_up) {
                went_team = true;
                potts_announce(sh, cl, kPottsLevels, C - f, C, level, c0, cn, t);
                uint32_t lo = C - f, hi = C;
                bool finished = false;
                potts_team_levels<DIM>(p, sh, cl, lo, hi, level, c0, tlo, thi, &finished);
                C = hi;
                f = finished ? 0u : hi - lo;
                for (uint32_t k = threadIdx.x; k < f && k < kLocalFrontierCap; k += blockDim.x)
                    sh.front[cur][k] = __ldcg(p.list + lo + k);
                if (t0) sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
                __syncthreads();
                continue;
            }
            const uint32_t nxt = cur ^ 1u;
            const uint32_t fbase = C - f;
            unsigned int *cnt = &sh.cnt[level % 3];
            if (t0) sh.cnt[(level + 1) % 3] = 0;
            for (uint32_t b = warp * 32u; b < f; b += nwarps * 32u) {
                const uint32_t k = b + lane;
                Neighbours<DIM> nb;
                uint32_t won = 0;
                if (k < f) {
                    const uint32_t packed =
                        k < kLocalFrontierCap ? sh.front[cur][k] : __ldcg(p.list + fbase + k);
                    won = potts_expand<DIM>(p, packed, c0, tlo, thi, nb);
                }
                uint32_t pos = warp_reserve(cnt, __popc(won));
#pragma unroll
                for (int s = 0; s < 2 * DIM; ++s) {
                    if (won & (1u << s)) {
                        const uint32_t gpos = C + pos;
                        if (gpos < p.g.N) p.list[gpos] = nb.packed[s];
                        else raise_status(ctl, WOLFF_EINVAL, 0xE3u);
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
        long long dE = 0;
        if (went_team || (has_team && C > kLocalListCap)) {
            potts_announce(sh, cl, kPottsFinish, 0, C, level, c0, cn, t);
            dE = potts_team_finish<DIM>(p, sh, cl, C, c0, cn);
        } else {
            const bool in_shared = C <= kLocalListCap;
            long long acc = 0;
            for (uint32_t k = threadIdx.x; k < C; k += blockDim.x)
                acc += potts_boundary<DIM>(p, in_shared ? sh.list[k] : __ldcg(p.list + k), c0, cn);
            dE = block_sum(acc);
            __syncthreads();
            for (uint32_t k = threadIdx.x; k < C; k += blockDim.x) {
                uint32_t c[DIM];
                unpack<DIM>(in_shared ? sh.list[k] : __ldcg(p.list + k), c);
                potts_flip(p.spins, site_index<DIM>(p.g, c), c0, cn);
                p.list[k] = kEmptySlot;
            }
        }
        if (t0) {
            E += dE;
            N0 += (long long)C * ((long long)(cn == 0) - (long long)(c0 == 0));
            total_C += C;
            last_C = C;
            last_levels = level;
            if (p.records) {
                wolff_record r;
                r.C = C;
                r.levels = level;
                r.E_bond = E;
                r.M = N0;
                p.records[u] = r;
            }
        }
        __syncthreads();
    }
    if (t0) {
        ctl->E = E;
        ctl->M = N0;
        ctl->total_C = total_C;
        ctl->last_C = last_C;
        ctl->last_levels = last_levels;
        ctl->t = p.t0 + p.n;
        ctl->st_updates += p.n;
        ctl->st_end_ns = global_ns();
    }
    if (has_team) {
        potts_announce(sh, cl, kPottsExit, 0, 0, 0, 0, 0, 0);
        cl.sync();
    }
}

template <int DIM>
__global__ void __launch_bounds__(512, 1) k_potts_team(StepParams p) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ PottsShared sh;
    if (cl.block_rank() != 0) {
        potts_worker<DIM>(p, sh, cl);
        return;
    }
    potts_leader<DIM>(p, sh, cl);
}

// Initial colours: floor(x q / 2^32), x = lane 0 of Philox(i, 0, 0, 2).
__global__ void k_potts_init(uint8_t *spins, uint32_t N, uint32_t q, uint32_t k0, uint32_t k1) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const Philox4 r = philox4x32_10(i, 0u, 0u, kTagInit, k0, k1);
        spins[i] = (uint8_t)(((unsigned long long)r.v[0] * q) >> 32);
    }
}

// Full recount: satisfied forward bonds and colour-0 sites (rows along x).
template <int DIM>
__global__ void k_potts_measure(const uint8_t *spins, Geometry g, DevCtl *ctl) {
    const uint32_t rows = g.N / g.L;
    long long e = 0, z = 0;
    for (uint32_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const uint32_t y = row % g.L;
        const uint32_t base = row * g.L;
        const uint32_t yup = (y + 1 == g.L) ? base + g.L - g.LL : base + g.L;
        uint32_t zup = 0;
        if (DIM == 3) {
            const uint32_t zz = row / g.L;
            zup = (zz + 1 == g.L) ? base + g.LL - g.N : base + g.LL;
        }
        for (uint32_t x = threadIdx.x; x < g.L; x += blockDim.x) {
            const uint32_t ci = spins[base + x] & kColourMask;
            const uint32_t xr = (x + 1 == g.L) ? 0 : x + 1;
            e += (ci == (spins[base + xr] & kColourMask)) + (ci == (spins[yup + x] & kColourMask));
            if (DIM == 3) e += ci == (spins[zup + x] & kColourMask);
            z += ci == 0;
        }
    }
    e = block_sum(e);
    z = block_sum(z);
    if (threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_E), (unsigned long long)e);
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_M), (unsigned long long)z);
    }
}

__global__ void k_potts_check(const uint8_t *spins, uint32_t N, uint32_t q, DevCtl *ctl) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        if (spins[i] >= q) raise_status(ctl, WOLFF_EINVAL, i);
}

__global__ void k_zero_full2(DevCtl *ctl) {
    ctl->full_E = 0;
    ctl->full_M = 0;
}

__global__ void k_full_to_chain2(DevCtl *ctl) {
    ctl->E = ctl->full_E;
    ctl->M = ctl->full_M;
}

unsigned grid_cap(unsigned long long work, unsigned long long cap) {
    unsigned long long b = work < cap ? work : cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_potts_init(uint8_t *spins, Geometry g, uint32_t q, uint32_t k0, uint32_t k1,
                              cudaStream_t s) {
    k_potts_init<<<grid_cap((g.N + 255) / 256, 4096), 256, 0, s>>>(spins, g.N, q, k0, k1);
    return cudaGetLastError();
}

cudaError_t launch_potts_measure(int dim, const uint8_t *spins, Geometry g, DevCtl *ctl,
                                 int set_chain, cudaStream_t s) {
    k_zero_full2<<<1, 1, 0, s>>>(ctl);
    const unsigned blocks = grid_cap(g.N / g.L, 8192), threads = g.L >= 256 ? 256 : 64;
    if (dim == 2)
        k_potts_measure<2><<<blocks, threads, 0, s>>>(spins, g, ctl);
    else
        k_potts_measure<3><<<blocks, threads, 0, s>>>(spins, g, ctl);
    if (set_chain) k_full_to_chain2<<<1, 1, 0, s>>>(ctl);
    return cudaGetLastError();
}

cudaError_t launch_potts_check(const uint8_t *spins, uint32_t N, uint32_t q, DevCtl *ctl,
                               cudaStream_t s) {
    k_potts_check<<<grid_cap((N + 255) / 256, 4096), 256, 0, s>>>(spins, N, q, ctl);
    return cudaGetLastError();
}

cudaError_t launch_potts_team(int dim, const StepParams &p, int cluster_size, int threads,
                              cudaStream_t s) {
    const void *fn = dim == 2 ? reinterpret_cast<const void *>(&k_potts_team<2>)
                              : reinterpret_cast<const void *>(&k_potts_team<3>);
    if (cluster_size > 8) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster_size);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster_size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {const_cast<StepParams *>(&p)};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace wolff
