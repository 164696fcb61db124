// wolff_team.cu -- the Wolff update run by a thread-block cluster ("team").
//
// One cluster of CS CTAs owns one lattice (a job) for the whole launch and
// runs its n updates.  Clusters never wait on one another, so a launch may
// hold any number of jobs -- one lattice (the plain form) or hundreds of
// independent replicas (the batched form) -- and the hardware schedules the
// clusters as SMs free up.  Inside a team:
//   - rank 0 (the leader) grows small wave fronts alone, with __syncthreads
//     as the level barrier and the front in shared memory (the on-GPU form of
//     the paper's hybrid, section 6);
//   - a front above t_up is expanded by all CTAs of the cluster, each taking
//     a stride of list[lo, hi); new sites get their list slots from counters
//     in the leader's shared memory (distributed shared memory atomics) and
//     levels are separated by the cluster barrier (barrier.cluster, release/
//     acquire at cluster scope), the GB300 hardware replacement of the
//     paper's quasi-block synchronisation (section 3).
// The worker CTAs of a team block in the cluster barrier while the leader
// works alone; every CTA of a cluster executes the same sequence of cluster
// barriers (the leader announces each team phase in its shared memory before
// the barrier that starts it), so the hardware barrier always completes.  The
// workers read the leader's shared memory remotely, so the team leaves the
// kernel only after a last cluster barrier that follows every such read.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "wolff_device.cuh"

namespace cg = cooperative_groups;

namespace wolff {

namespace {

enum : unsigned int { kTeamLevels = 1, kTeamFinish = 2, kTeamExit = 3 };

struct TeamShared {
    uint32_t front[2][kLocalFrontierCap];
    uint32_t list[kLocalListCap];
    unsigned int cnt[3];        // level append counters (the leader's are the team's)
    unsigned int sig0bit;
    unsigned int cmd[8];        // kind, lo, hi, level, sig0bit, t_lo, t_hi
    unsigned long long dE;      // team boundary sum (leader's copy)
};

// All CTAs of the team: expand level after level from list[lo, hi) until the
// next front is empty (*finished) or has t_down sites or fewer.
template <int DIM>
__device__ __forceinline__ void team_levels(const StepParams &p, TeamShared &sh,
                                            cg::cluster_group &cl, uint32_t &lo, uint32_t &hi,
                                            uint32_t &level, uint32_t sig0bit, uint32_t tlo,
                                            uint32_t thi, bool *finished) {
    TeamShared *lead = cl.map_shared_rank(&sh, 0);
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
            if (k < hi) won = expand_site<DIM>(p, __ldcg(p.list + k), sig0bit, tlo, thi, nb);
            uint32_t pos = hi + warp_reserve(cnt, __popc(won));
#pragma unroll
            for (int s = 0; s < 2 * DIM; ++s) {
                if (won & (1u << s)) {
                    if (pos < p.g.N) p.list[pos] = nb.packed[s];
                    else raise_status(p.ctl, WOLFF_EINVAL, 0xD0u);
                    ++pos;
                }
            }
        }
        cl.sync();
        uint32_t added = *reinterpret_cast<volatile unsigned int *>(cnt);
        ++level;
        if (added > p.g.N - hi) {   // cannot happen: every site joins at most once
            if (rank == 0 && threadIdx.x == 0) raise_status(p.ctl, WOLFF_EINVAL, 0xD1u);
            added = 0;
        }
        lo = hi;
        hi += added;
        if (added == 0 || added <= p.t_down) {
            *finished = added == 0;
            // every CTA has read the count before the leader reuses the counters
            cl.sync();
            return;
        }
    }
}

// All CTAs of the team: boundary sum over list[0, C), then unmark.  Returns
// the sum in the leader's thread 0.
template <int DIM>
__device__ __forceinline__ long long team_finish(const StepParams &p, TeamShared &sh,
                                                 cg::cluster_group &cl, uint32_t C,
                                                 uint32_t sig0bit) {
    TeamShared *lead = cl.map_shared_rank(&sh, 0);
    const unsigned int rank = cl.block_rank(), cs = cl.num_blocks();
    const uint32_t tid = rank * blockDim.x + threadIdx.x, nt = cs * blockDim.x;
    long long acc = 0;
    for (uint32_t k = tid; k < C; k += nt) {
        uint32_t i;
        acc += boundary_term<DIM>(p, __ldcg(p.list + k), sig0bit, &i);
    }
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
        unmark_site(p.spins, site_index<DIM>(p.g, c), sig0bit);
        p.list[k] = kEmptySlot;
    }
    cl.sync();
    return dE;
}

template <int DIM>
__device__ void team_worker(const StepParams &p, TeamShared &sh, cg::cluster_group &cl) {
    TeamShared *lead = cl.map_shared_rank(&sh, 0);
    while (true) {
        cl.sync();   // the leader has announced the next phase
        const volatile unsigned int *cmd = lead->cmd;
        const unsigned int kind = cmd[0];
        uint32_t lo = cmd[1], hi = cmd[2], level = cmd[3];
        const uint32_t sig0bit = cmd[4], tlo = cmd[5], thi = cmd[6];
        if (kind == kTeamLevels) {
            bool finished = false;
            team_levels<DIM>(p, sh, cl, lo, hi, level, sig0bit, tlo, thi, &finished);
        } else if (kind == kTeamFinish) {
            team_finish<DIM>(p, sh, cl, hi, sig0bit);
        } else {
            // the leader's shared memory (read above) must outlive every
            // remote access: leave together, after one more cluster barrier
            cl.sync();
            return;
        }
    }
}

// Leader: announce a team phase, then start it with the cluster barrier.
__device__ __forceinline__ void announce(TeamShared &sh, cg::cluster_group &cl, unsigned int kind,
                                         uint32_t lo, uint32_t hi, uint32_t level,
                                         uint32_t sig0bit, unsigned long long t) {
    if (threadIdx.x == 0) {
        sh.cmd[0] = kind;
        sh.cmd[1] = lo;
        sh.cmd[2] = hi;
        sh.cmd[3] = level;
        sh.cmd[4] = sig0bit;
        sh.cmd[5] = (uint32_t)t;
        sh.cmd[6] = (uint32_t)(t >> 32);
        sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
    }
    cl.sync();
}

template <int DIM>
__device__ void team_leader(const StepParams &p, TeamShared &sh, cg::cluster_group &cl) {
    DevCtl *ctl = p.ctl;
    const bool t0 = threadIdx.x == 0;
    const bool has_team = cl.num_blocks() > 1;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long E = 0, M = 0;
    unsigned long long total_C = 0;
    uint32_t last_C = 0, last_levels = 0;
    unsigned long long st_local = 0, st_team = 0, ns_local = 0, ns_team = 0, ns_finish = 0;
    unsigned long long handoffs = 0, team_fin = 0;
    if (t0) {
        ctl->st_start_ns = global_ns();
        E = ctl->E;
        M = ctl->M;
        total_C = ctl->total_C;
        last_C = ctl->last_C;
        last_levels = ctl->last_levels;
        sh.dE = 0;
    }
    for (unsigned long long u = 0; u < p.n; ++u) {
        const unsigned long long t = p.t0 + u;
        const uint32_t tlo = (uint32_t)t, thi = (uint32_t)(t >> 32);
        unsigned long long clk = 0;
        if (t0) {
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
            clk = global_ns();
        }
        __syncthreads();
        const uint32_t sig0bit = sh.sig0bit;
        uint32_t C = 1, f = 1, level = 0, cur = 0;
        bool went_team = false;
        while (f > 0) {
            if (has_team && f > p.t_up) {
                went_team = true;
                unsigned long long g0 = 0;
                if (t0) {
                    g0 = global_ns();
                    ns_local += g0 - clk;
                    ++handoffs;
                }
                announce(sh, cl, kTeamLevels, C - f, C, level, sig0bit, t);
                uint32_t lo = C - f, hi = C, lv0 = level;
                bool finished = false;
                team_levels<DIM>(p, sh, cl, lo, hi, level, sig0bit, tlo, thi, &finished);
                C = hi;
                f = finished ? 0u : hi - lo;
                for (uint32_t k = threadIdx.x; k < f && k < kLocalFrontierCap; k += blockDim.x)
                    sh.front[cur][k] = __ldcg(p.list + lo + k);
                if (t0) {
                    sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
                    st_team += level - lv0;
                    clk = global_ns();
                    ns_team += clk - g0;
                }
                __syncthreads();
                continue;
            }
            // one level on the leader alone; a front larger than the shared
            // buffer is read from the cluster list, which this CTA wrote
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
                    won = expand_site<DIM>(p, packed, sig0bit, tlo, thi, nb);
                }
                uint32_t pos = warp_reserve(cnt, __popc(won));
#pragma unroll
                for (int s = 0; s < 2 * DIM; ++s) {
                    if (won & (1u << s)) {
                        const uint32_t gpos = C + pos;
                        if (gpos < p.g.N) p.list[gpos] = nb.packed[s];
                        else raise_status(ctl, WOLFF_EINVAL, 0xD3u);
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
        if (went_team || (has_team && C > p.t_up * 4u && C > kLocalListCap)) {
            if (t0) ++team_fin;
            announce(sh, cl, kTeamFinish, 0, C, level, sig0bit, t);
            dE = team_finish<DIM>(p, sh, cl, C, sig0bit);
        } else {
            // the leader closes the cluster alone
            const bool in_shared = C <= kLocalListCap;
            long long acc = 0;
            for (uint32_t k = threadIdx.x; k < C; k += blockDim.x) {
                uint32_t i;
                acc += boundary_term<DIM>(p, in_shared ? sh.list[k] : __ldcg(p.list + k), sig0bit,
                                          &i);
            }
            dE = block_sum(acc);
            __syncthreads();
            for (uint32_t k = threadIdx.x; k < C; k += blockDim.x) {
                uint32_t c[DIM];
                unpack<DIM>(in_shared ? sh.list[k] : __ldcg(p.list + k), c);
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
            ns_finish += global_ns() - f0;
        }
        __syncthreads();
    }
    if (t0) {
        ctl->E = E;
        ctl->M = M;
        ctl->total_C = total_C;
        ctl->last_C = last_C;
        ctl->last_levels = last_levels;
        ctl->t = p.t0 + p.n;
        ctl->st_updates += p.n;
        ctl->st_levels_local += st_local;
        ctl->st_levels_grid += st_team;
        ctl->st_ns_local += ns_local;
        ctl->st_ns_grid += ns_team;
        ctl->st_ns_finish += ns_finish;
        ctl->st_handoffs += handoffs;
        ctl->st_grid_finishes += team_fin;
        ctl->st_end_ns = global_ns();
    }
    if (has_team) {
        announce(sh, cl, kTeamExit, 0, 0, 0, 0, 0);
        cl.sync();   // no CTA of the team exits while another may still read its shared memory
    }
}

template <int DIM>
__global__ void __launch_bounds__(512, 1) k_team(StepParams single, const StepParams *table) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ TeamShared sh;
    const unsigned int job = blockIdx.x / cl.num_blocks();
    const StepParams p = table ? table[job] : single;
    if (cl.block_rank() != 0) {
        team_worker<DIM>(p, sh, cl);
        return;
    }
    team_leader<DIM>(p, sh, cl);
}

}  // namespace

const void *team_kernel(int dim) {
    return dim == 2 ? reinterpret_cast<const void *>(&k_team<2>)
                    : reinterpret_cast<const void *>(&k_team<3>);
}

cudaError_t launch_team(int dim, const StepParams &single, const StepParams *d_table, int njobs,
                        int cluster_size, int threads, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    const void *fn = team_kernel(dim);
    if (cluster_size > 8) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(njobs * cluster_size));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster_size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {const_cast<StepParams *>(&single), const_cast<StepParams **>(&d_table)};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace wolff
