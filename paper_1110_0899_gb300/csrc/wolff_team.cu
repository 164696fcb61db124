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

enum : unsigned int { kTeamLevels = 1, kTeamFinish = 2, kTeamExit = 3, kTeamBurst = 4 };

// ---- burst mode --------------------------------------------------------------
// While clusters are small, consecutive updates rarely touch the same sites.
// The leader then grows up to one update per warp at once, all on the same
// lattice, without claiming anything (each warp keeps its cluster in a
// shared-memory hash set), and afterwards commits, in order, the longest
// prefix whose updates read no site that an earlier update of the prefix
// flips.  Update t+j reads its members and their neighbours; if none of them
// was flipped by updates t..t+j-1, it sees exactly the lattice the serial
// chain would show it, so every committed update is the serial one -- the
// same component, level count, boundary sum and record.  The first update that
// conflicts, or whose cluster outgrows kBurstCap, is left for the ordinary path.
constexpr int kBurstMaxWarps = 16;
constexpr uint32_t kBurstCap = 64;          // members per speculative update (128 at <= 8 warps)
constexpr uint32_t kBurstMapSlots = 2048;   // flipped-site map of the whole burst
constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;

struct TeamShared {
    uint32_t front[2][kLocalFrontierCap];
    uint32_t list[kLocalListCap];
    unsigned int cnt[3];        // level append counters (the leader's are the team's)
    unsigned int sig0bit;
    unsigned int cmd[8];        // kind, lo, hi, level, sig0bit, t_lo, t_hi
    unsigned long long dE;      // team boundary sum (leader's copy)
    // burst mode (leader only): per-warp results and the commit cut
    int bres[kBurstMaxWarps][4];  // |C| (or -1 when too big), levels, dE_bond, sig0bit
    unsigned int bcut;
    unsigned int bflag;
    unsigned int bstop;
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
__device__ uint32_t team_burst(const StepParams &p, TeamShared &sh, cg::cluster_group &cl,
                               unsigned long long u0, uint32_t nb, long long &E, long long &M,
                               unsigned long long &total_C, uint32_t &last_C,
                               uint32_t &last_levels);

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
        } else if (kind == kTeamBurst) {
            long long E = 0, M = 0;
            unsigned long long tc = 0;
            uint32_t lc = 0, ll = 0;
            team_burst<DIM>(p, sh, cl, ((unsigned long long)hi << 32) | lo, level, E, M, tc, lc,
                            ll);
        } else {
            // the leader's shared memory (read above) must outlive every
            // remote access: leave together, after one more cluster barrier
            cl.sync();
            return;
        }
    }
}


__device__ __forceinline__ uint32_t burst_hash(uint32_t key, uint32_t slots) {
    return (key * 0x9E3779B1u) >> (32 - __ffs(slots) + 1);
}

// Inserts key into an open-addressing set of `slots` entries (power of two).
// Returns 1 if newly inserted, 0 if present, -1 if the set is full.
__device__ __forceinline__ int burst_insert(uint32_t *set, uint32_t slots, uint32_t key) {
    uint32_t h = burst_hash(key, slots);
    for (uint32_t probe = 0; probe < slots; ++probe) {
        const uint32_t prev = atomicCAS(set + h, kEmptyKey, key);
        if (prev == kEmptyKey) return 1;
        if (prev == key) return 0;
        h = (h + 1) & (slots - 1);
    }
    return -1;
}

__device__ __forceinline__ bool burst_contains(const uint32_t *set, uint32_t slots, uint32_t key) {
    uint32_t h = burst_hash(key, slots);
    for (uint32_t probe = 0; probe < slots; ++probe) {
        const uint32_t v = set[h];
        if (v == key) return true;
        if (v == kEmptyKey) return false;
        h = (h + 1) & (slots - 1);
    }
    return false;
}

// Owner CTA of a site in the team's distributed flipped-site map.
__device__ __forceinline__ uint32_t burst_owner(uint32_t site, uint32_t cs) {
    return ((site * 0x85EBCA6Bu) >> 16) & (cs - 1u);
}

// All CTAs of the team: grow, check and commit up to nb consecutive updates
// starting at p.t0 + u0, update u0 + g on warp g % W of CTA g / W (W warps per
// CTA).  The map "lowest update index that flips a site" is spread over the
// CTAs' shared memory (each site has an owner CTA) and reached through
// distributed shared memory; cluster barriers separate growth, insertion,
// checking and commit.  Returns how many updates were committed (0 when the
// first one is too big); the leader's thread 0 advances the chain state and
// writes their records.
template <int DIM>
__device__ uint32_t team_burst(const StepParams &p, TeamShared &sh, cg::cluster_group &cl,
                               unsigned long long u0, uint32_t nb, long long &E, long long &M,
                               unsigned long long &total_C, uint32_t &last_C,
                               uint32_t &last_levels) {
    const uint32_t W = min((uint32_t)(blockDim.x >> 5), (uint32_t)kBurstMaxWarps);
    const uint32_t rank = cl.block_rank(), cs = cl.num_blocks();
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t g = rank * W + warp;
    const bool active = warp < W && g < nb;
    TeamShared *lead = cl.map_shared_rank(&sh, 0);
    uint32_t *raw = &sh.front[0][0];                 // 8192 words, free outside growth
    uint32_t *map_key = raw;                         // kBurstMapSlots
    uint32_t *map_val = raw + kBurstMapSlots;        // kBurstMapSlots
    // a CTA with 8 warps or fewer gives each of them room for 128 members
    const uint32_t cap = W <= 8 ? 2 * kBurstCap : kBurstCap, hslots = 2 * cap;
    uint32_t *mine = raw + 2 * kBurstMapSlots + (warp % kBurstMaxWarps) * (cap + hslots);
    uint32_t *members = mine, *hset = mine + cap;
    for (uint32_t k = threadIdx.x; k < kBurstMapSlots; k += blockDim.x) {
        map_key[k] = kEmptyKey;
        map_val[k] = 0xFFFFFFFFu;
    }
    bool too_big = false;
    uint32_t n = 0;
    // ---- grow
    if (active) {
        for (uint32_t k = lane; k < hslots; k += 32) hset[k] = kEmptyKey;
        __syncwarp();
        const unsigned long long t = p.t0 + u0 + g;
        const uint32_t tlo = (uint32_t)t, thi = (uint32_t)(t >> 32);
        const uint32_t i0 = seed_site(p, t);
        const uint32_t sig0bit = __ldcg(p.spins + i0) & 1u;
        if (lane == 0) {
            burst_insert(hset, hslots, i0);
            members[0] = pack_index<DIM>(p.g, i0);
        }
        __syncwarp();
        n = 1;
        uint32_t lo = 0, levels = 0;
        while (lo < n && !too_big) {
            const uint32_t hi = n;
            for (uint32_t b = lo; b < hi; b += 32) {
                const uint32_t k = b + lane;
                Neighbours<DIM> nb2;
                uint32_t fresh = 0;
                bool full = false;
                if (k < hi) {
                    uint32_t i;
                    neighbours<DIM>(p.g, members[k], &i, nb2);
                    uint8_t v[2 * DIM];
#pragma unroll
                    for (int s = 0; s < 2 * DIM; ++s) v[s] = __ldcg(p.spins + nb2.idx[s]);
                    uint32_t owners[DIM + 1];
                    owners[0] = i;
#pragma unroll
                    for (int d = 0; d < DIM; ++d) owners[d + 1] = nb2.idx[2 * d + 1];
                    Philox4 draw[DIM + 1];
                    philox4x32_10_lanes<DIM + 1>(owners, tlo, thi, kTagBond, p.key0, p.key1, draw);
#pragma unroll
                    for (int s = 0; s < 2 * DIM; ++s) {
                        const int d = s >> 1;
                        const uint32_t r = (s & 1) ? draw[d + 1].v[d] : draw[0].v[d];
                        if ((uint32_t)(v[s] & 1u) == sig0bit && (unsigned long long)r < p.thr) {
                            const int ins = burst_insert(hset, hslots, nb2.idx[s]);
                            if (ins > 0) fresh |= 1u << s;
                            if (ins < 0) full = true;
                        }
                    }
                }
                const uint32_t cnt = __popc(fresh);
                uint32_t incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFullMask, incl, o);
                    if (lane >= o) incl += y;
                }
                const uint32_t total = __shfl_sync(kFullMask, incl, 31);
                uint32_t pos = n + incl - cnt;
#pragma unroll
                for (int s = 0; s < 2 * DIM; ++s) {
                    if (fresh & (1u << s)) {
                        if (pos < cap) members[pos] = nb2.packed[s];
                        ++pos;
                    }
                }
                n += total;
                if (__any_sync(kFullMask, full) || n > cap) too_big = true;
            }
            __syncwarp();
            ++levels;
            lo = hi;
        }
        int dE = 0;
        if (!too_big) {
            for (uint32_t k = lane; k < n; k += 32) {
                uint32_t i;
                Neighbours<DIM> nb2;
                neighbours<DIM>(p.g, members[k], &i, nb2);
#pragma unroll
                for (int s = 0; s < 2 * DIM; ++s) {
                    if (burst_contains(hset, hslots, nb2.idx[s])) continue;
                    const uint32_t cur = __ldcg(p.spins + nb2.idx[s]) & 1u;
                    dE += (cur == sig0bit) ? -1 : 1;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dE += __shfl_down_sync(kFullMask, dE, o);
        }
        if (lane == 0) {
            sh.bres[warp][0] = too_big ? -1 : (int)n;
            sh.bres[warp][1] = (int)levels;
            sh.bres[warp][2] = dE;
            sh.bres[warp][3] = (int)sig0bit;
            if (too_big) atomicMin(&lead->bcut, g);
        }
    }
    cl.sync();   // every CTA has grown its updates and cleared its part of the map
    // ---- the lowest update index that flips each site, in the owner CTA's map
    if (active && !too_big) {
        bool lost = false;
        for (uint32_t k = lane; k < n; k += 32) {
            uint32_t c[DIM];
            unpack<DIM>(members[k], c);
            const uint32_t site = site_index<DIM>(p.g, c);
            uint32_t *rraw = cl.map_shared_rank(raw, burst_owner(site, cs));
            uint32_t h = burst_hash(site * 0x9E3779B1u + 0x7F4A7C15u, kBurstMapSlots);
            bool placed = false;
            for (uint32_t probe = 0; probe < kBurstMapSlots; ++probe) {
                const uint32_t prev = atomicCAS(rraw + h, kEmptyKey, site);
                if (prev == kEmptyKey || prev == site) {
                    atomicMin(rraw + kBurstMapSlots + h, g);
                    placed = true;
                    break;
                }
                h = (h + 1) & (kBurstMapSlots - 1);
            }
            if (!placed) lost = true;
        }
        // a map too full to record a flip makes the update unsafe to commit
        if (__any_sync(kFullMask, lost) && lane == 0) atomicMin(&lead->bcut, g);
    }
    cl.sync();
    // ---- update g conflicts if it read a site flipped by an earlier update
    if (active && !too_big) {
        bool conflict = false;
        for (uint32_t k = lane; k < n && !conflict; k += 32) {
            uint32_t i;
            Neighbours<DIM> nb2;
            neighbours<DIM>(p.g, members[k], &i, nb2);
            uint32_t probe_sites[2 * DIM + 1];
            probe_sites[0] = i;
#pragma unroll
            for (int s = 0; s < 2 * DIM; ++s) probe_sites[s + 1] = nb2.idx[s];
#pragma unroll
            for (int q = 0; q < 2 * DIM + 1; ++q) {
                const uint32_t site = probe_sites[q];
                const uint32_t *rraw = cl.map_shared_rank(raw, burst_owner(site, cs));
                uint32_t h = burst_hash(site * 0x9E3779B1u + 0x7F4A7C15u, kBurstMapSlots);
                for (uint32_t probe = 0; probe < kBurstMapSlots; ++probe) {
                    const uint32_t key = rraw[h];
                    if (key == site) {
                        if (rraw[kBurstMapSlots + h] < g) conflict = true;
                        break;
                    }
                    if (key == kEmptyKey) break;
                    h = (h + 1) & (kBurstMapSlots - 1);
                }
            }
        }
        if (__any_sync(kFullMask, conflict) && lane == 0) atomicMin(&lead->bcut, g);
    }
    cl.sync();
    const uint32_t cut = *reinterpret_cast<volatile unsigned int *>(&lead->bcut);
    // ---- commit updates [0, cut): flip their members (both bits)
    if (active && g < cut) {
        const uint8_t v = sh.bres[warp][3] ? 0x00 : 0x03;
        for (uint32_t k = lane; k < n; k += 32) {
            uint32_t c[DIM];
            unpack<DIM>(members[k], c);
            p.spins[site_index<DIM>(p.g, c)] = v;
        }
    }
    if (rank == 0 && cut > 0) {
        // records of the committed updates in parallel: a scan of the energy
        // and magnetisation steps over the leader CTA
        __shared__ long long s_e[512], s_m[512];
        __shared__ unsigned long long s_c[512];
        __shared__ long long s_base[2];
        const uint32_t j = threadIdx.x;
        int res[4] = {0, 0, 0, 0};
        if (j < cut) {
            const TeamShared *src = cl.map_shared_rank(&sh, j / W);
#pragma unroll
            for (int q = 0; q < 4; ++q) res[q] = src->bres[j % W][q];
        }
        s_e[j] = j < cut ? 2LL * res[2] : 0;
        s_m[j] = j < cut ? (res[3] ? -2LL : 2LL) * res[0] : 0;
        s_c[j] = j < cut ? (unsigned long long)res[0] : 0;
        if (j == 0) {
            s_base[0] = E;
            s_base[1] = M;
        }
        __syncthreads();
        for (uint32_t off = 1; off < cut; off <<= 1) {
            const long long ve = j >= off ? s_e[j - off] : 0;
            const long long vm = j >= off ? s_m[j - off] : 0;
            const unsigned long long vc = j >= off ? s_c[j - off] : 0;
            __syncthreads();
            s_e[j] += ve;
            s_m[j] += vm;
            s_c[j] += vc;
            __syncthreads();
        }
        if (j < cut && p.records) {
            wolff_record r;
            r.C = (uint32_t)res[0];
            r.levels = (uint32_t)res[1];
            r.E_bond = s_base[0] + s_e[j];
            r.M = s_base[1] + s_m[j];
            p.records[u0 + j] = r;
        }
        if (j == cut - 1) {
            s_base[0] += s_e[j];
            s_base[1] += s_m[j];
            s_c[511] = s_c[j];
            s_e[511] = res[0];
            s_m[511] = res[1];
        }
        __syncthreads();
        if (j == 0) {
            E = s_base[0];
            M = s_base[1];
            total_C += s_c[511];
            last_C = (uint32_t)s_e[511];
            last_levels = (uint32_t)s_m[511];
        }
    }
    cl.sync();   // results read and commits done before anything is reused
    return cut;
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
    // burst policy (thread 0 decides, the CTA follows): bursts run while the
    // recent clusters are small; a cluster too big for a burst pauses them
    unsigned int cooldown = 0, fail_streak = 0, skip_next = 0;
    unsigned long long bursts_done = 0, burst_calls = 0;
    const unsigned long long launch_t0 = global_ns();
    unsigned long long u = 0;
    for (; u < p.n; ++u) {
        if (p.budget_ns && u > 0) {   // a time-budgeted job stops at an update boundary
            if (t0) sh.bstop = (global_ns() - launch_t0 > p.budget_ns) ? 1u : 0u;
            __syncthreads();
            if (sh.bstop) break;
        }
        if (p.burst && p.n - u >= 2) {
            // a burst cut short by an update too big for it leaves that update
            // to the ordinary path directly
            if (t0) sh.bflag = (cooldown == 0 && !skip_next) ? 1u : 0u;
            __syncthreads();
            if (sh.bflag) {
                const uint32_t W = min((uint32_t)(blockDim.x >> 5), (uint32_t)kBurstMaxWarps);
                const uint32_t nb =
                    (uint32_t)min((unsigned long long)(W * cl.num_blocks()), p.n - u);
                if (t0) sh.bcut = nb;
                if (has_team)
                    announce(sh, cl, kTeamBurst, (uint32_t)u, (uint32_t)(u >> 32), nb, 0, 0);
                else
                    __syncthreads();
                const uint32_t c = team_burst<DIM>(p, sh, cl, u, nb, E, M, total_C, last_C,
                                                   last_levels);
                if (t0) {
                    bursts_done += c;
                    ++burst_calls;
                    if (c > 0 && c < nb) {
                        const TeamShared *src = cl.map_shared_rank(&sh, c / W);
                        skip_next = src->bres[c % W][0] < 0 ? 1u : 0u;
                    }
                    // back off only while bursts keep failing at their first
                    // update (the large-cluster regime): 0, 1, 3, ..., 63
                    if (c == 0) {
                        fail_streak = min(fail_streak + 1u, 7u);
                        cooldown = (1u << (fail_streak - 1u)) - 1u;
                    } else {
                        fail_streak = 0;
                    }
                }
                if (c > 0) {
                    u += c - 1;
                    continue;
                }
            } else if (t0) {
                if (skip_next) skip_next = 0;
                else --cooldown;
            }
        }
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
        ctl->t = p.t0 + u;
        ctl->st_updates += u;
        ctl->st_levels_local += st_local;
        ctl->st_levels_grid += st_team;
        ctl->st_ns_local += ns_local;
        ctl->st_ns_grid += ns_team;
        ctl->st_ns_finish += ns_finish;
        ctl->st_handoffs += handoffs;
        ctl->st_grid_finishes += team_fin;
        ctl->st_burst_updates += bursts_done;
        ctl->st_bursts += burst_calls;
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
