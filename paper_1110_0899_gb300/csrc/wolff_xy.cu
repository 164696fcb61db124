// wolff_xy.cu -- the XY embedded-cluster update on a team.
//
// Section 6 of the paper names the XY model as the next extension of its GPU
// cluster growth.  H = -J sum_<ij> cos(theta_i - theta_j), updated by
// Wolff's embedded Ising cluster: update t draws a seed site (lane 0 of the
// seed draw) and a reflection angle phi (lane 1); a bond <ij> is active with
// p = 1 - exp(-2K (r.s_i)(r.s_j)) when (r.s_i)(r.s_j) > 0, judged on the
// pre-update angles with the same bond words as the Ising update; every
// member of the seed's component is reflected, theta -> pi + 2 phi - theta.
//
// Exact integer arithmetic (the header states the definitions): angles are
// integers in units of 2 pi / 65536, projections come from a fixed-point
// cosine table, and e^-y of the bond test is evaluated by Cody-Waite range
// reduction and a Taylor series (Cody & Waite, Software Manual for the
// Elementary Functions, 1980) in correctly rounded double intrinsics in a
// fixed order, so every bond decision is a function of integers only.
//
// Site word: bits 0..15 angle, bit 31 "claimed in this update".  Angles do
// not change while a cluster grows, so the bond test never depends on who
// claimed what first; the claim is one idempotent atomicOr of bit 31.  The
// boundary sums (E, Mx, My) read the claim bits of the neighbours, then the
// reflection writes each member's new angle and clears its bit.
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

constexpr uint32_t kXyMark = 0x80000000u;
constexpr uint32_t kXyAngle = 0xFFFFu;

enum : unsigned int { kXyLevels = 1, kXyFinish = 2, kXyExit = 3 };

struct XyShared {
    uint32_t front[2][kLocalFrontierCap];
    uint32_t list[kLocalListCap];
    unsigned int cnt[3];
    unsigned int phi;
    unsigned int cmd[8];          // kind, lo, hi, level, phi, -, t_lo, t_hi
    unsigned long long sum[3];    // team boundary sums (leader's copy)
    long long red[3][16];         // per-warp partial sums
};

// Fixed-point cos of angle a (units 2 pi / 65536) from the quarter-wave table.
__device__ __forceinline__ int32_t xy_cos(const int32_t *tab, uint32_t a) {
    a &= kXyAngle;
    const uint32_t q = a >> 14, r = a & 0x3FFFu;
    const int32_t v = __ldg(tab + ((q & 1u) ? 16384u - r : r));
    return (q == 1u || q == 2u) ? -v : v;
}

// e^-y, y >= 0: y = k ln2 + r, |r| <= ln2 / 2; e^-r by its Taylor series to
// degree 16 (Horner), then scaled by 2^-k.  ln 2 is split into a 32-bit head
// (k ln2_hi is exact) and the double tail.
__device__ __forceinline__ double xy_exp_neg(double y, const double *coef) {
    const double kInvLn2 = 0x1.71547652b82fep+0;
    const double kLn2Hi = 0x1.62e42feep-1;
    const double kLn2Lo = 0x1.a39ef35793c76p-33;
    if (!(y < 1000.0)) return 0.0;
    const double kd = floor(__dadd_rn(__dmul_rn(y, kInvLn2), 0.5));
    const double r = __dsub_rn(__dsub_rn(y, __dmul_rn(kd, kLn2Hi)), __dmul_rn(kd, kLn2Lo));
    const double m = -r;
    double s = __ldg(coef + 16);
#pragma unroll
    for (int n = 15; n >= 0; --n) s = __dadd_rn(__dmul_rn(s, m), __ldg(coef + n));
    return ldexp(s, -(int)kd);
}

// floor(2^32 (1 - e^-y)), y = kk * prod, for prod > 0; else 0.
__device__ __forceinline__ unsigned long long xy_threshold(long long prod, const StepParams &p) {
    if (prod <= 0) return 0ull;
    const double y = __dmul_rn(p.xy_kk, __ll2double_rn(prod));
    const double pr = __dsub_rn(1.0, xy_exp_neg(y, p.xy_coef));
    if (!(pr > 0.0)) return 0ull;
    if (pr >= 1.0) return 1ull << 32;
    return (unsigned long long)floor(__dmul_rn(pr, 4294967296.0));
}

// The bond test r < floor(2^32 (1 - e^-y)), decided first in single
// precision.  p_f = 1 - expf(-y_f) with y_f = float(kk) * float(prod):
// y_f = y (1 + e), |e| <= 3 * 2^-24, expf is within 2 ulp (CUDA programming
// guide, appendix on mathematical functions), and the subtraction rounds by
// at most 2^-24, so |p_f - p| < max_y (e^-y y 3 2^-24) + 2 * 2^-23 + 2^-24
// < 4e-7.  The bounds (p_f -+ m) 2^32 are rounded by at most 512 units of r
// and float(r) by at most 128, all far inside the margin m 2^32 = 8590
// units: r + 1 <= lower bound proves r < floor(p 2^32) (accept), r >= upper
// bound proves r >= floor(p 2^32) (reject).  Between the bounds (a few times
// 1e-6 of the tests) the double-precision path decides.  The fast path uses
// no double-precision operation.
constexpr float kXyMargin = 2.0e-6f;

__device__ __forceinline__ bool xy_bond_active(uint32_t r, long long prod, float kk_f,
                                               const StepParams &p) {
    if (prod <= 0) return false;
    const float yf = __fmul_rn(kk_f, __ll2float_rn(prod));
    const float pf = __fsub_rn(1.0f, expf(-yf));
    const float rf = __uint2float_rn(r);
    if (__fadd_rn(rf, 1.0f) <= __fmul_rn(__fsub_rn(pf, kXyMargin), 4294967296.0f)) return true;
    if (rf >= __fmul_rn(__fadd_rn(pf, kXyMargin), 4294967296.0f)) return false;
    return (unsigned long long)r < xy_threshold(prod, p);
}

__device__ __forceinline__ uint32_t xy_reflect(uint32_t theta, uint32_t phi) {
    return (32768u + 2u * phi - theta) & kXyAngle;
}

// Claims every unclaimed neighbour behind an active bond.  Returns the mask of
// neighbour slots won; nb receives their coordinates.
template <int DIM>
__device__ __forceinline__ uint32_t xy_expand(const StepParams &p, uint32_t packed, uint32_t phi,
                                              uint32_t tlo, uint32_t thi, Neighbours<DIM> &nb) {
    uint32_t *w = reinterpret_cast<uint32_t *>(p.spins);
    uint32_t i;
    neighbours<DIM>(p.g, packed, &i, nb);
    const uint32_t wi = __ldcg(w + i);
    uint32_t v[2 * DIM];
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) v[s] = __ldcg(w + nb.idx[s]);
    uint32_t owners[DIM + 1];
    owners[0] = i;
#pragma unroll
    for (int d = 0; d < DIM; ++d) owners[d + 1] = nb.idx[2 * d + 1];
    Philox4 draw[DIM + 1];
    philox4x32_10_lanes<DIM + 1>(owners, tlo, thi, kTagBond, p.key0, p.key1, draw);
    const long long si = xy_cos(p.xy_tab, (wi & kXyAngle) + 65536u - phi);
    const float kk_f = __double2float_rn(p.xy_kk);
    uint32_t want = 0;
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) {
        if (v[s] & kXyMark) continue;
        const int d = s >> 1;
        const uint32_t r = (s & 1) ? draw[d + 1].v[d] : draw[0].v[d];
        const long long sj = xy_cos(p.xy_tab, (v[s] & kXyAngle) + 65536u - phi);
        if (xy_bond_active(r, si * sj, kk_f, p)) want |= 1u << s;
    }
    unsigned int old[2 * DIM];
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) {
        old[s] = 0;
        if (want & (1u << s)) old[s] = atomicOr(w + nb.idx[s], kXyMark);
    }
    uint32_t won = 0;
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s)
        if ((want & (1u << s)) && !(old[s] & kXyMark)) won |= 1u << s;
    return won;
}

// Changes of E, Mx, My from reflecting one member: bonds to neighbours
// outside the cluster change; bonds inside keep their angle difference up to
// sign, and cos is even.
template <int DIM>
__device__ __forceinline__ void xy_boundary(const StepParams &p, uint32_t packed, uint32_t phi,
                                            long long acc[3]) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(p.spins);
    uint32_t i;
    Neighbours<DIM> nb;
    neighbours<DIM>(p.g, packed, &i, nb);
    const uint32_t th = __ldcg(w + i) & kXyAngle, nt = xy_reflect(th, phi);
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) {
        const uint32_t v = __ldcg(w + nb.idx[s]);
        if (v & kXyMark) continue;
        const uint32_t tj = v & kXyAngle;
        acc[0] += (long long)xy_cos(p.xy_tab, nt + 65536u - tj) -
                  xy_cos(p.xy_tab, th + 65536u - tj);
    }
    acc[1] += (long long)xy_cos(p.xy_tab, nt) - xy_cos(p.xy_tab, th);
    acc[2] += (long long)xy_cos(p.xy_tab, nt + 65536u - 16384u) -
              xy_cos(p.xy_tab, th + 65536u - 16384u);
}

__device__ __forceinline__ void xy_flip(const StepParams &p, uint32_t j, uint32_t phi) {
    uint32_t *w = reinterpret_cast<uint32_t *>(p.spins);
    w[j] = xy_reflect(__ldcg(w + j) & kXyAngle, phi);
}

// Block sums of three 64-bit values (every thread gets them).
__device__ __forceinline__ void xy_block_sum3(XyShared &sh, long long v[3]) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(kFullMask, v[q], o);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) sh.red[q][warp] = v[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        long long t = 0;
        for (uint32_t k = 0; k < nw; ++k) t += sh.red[q][k];
        v[q] = t;
    }
}

template <int DIM>
__device__ void xy_team_levels(const StepParams &p, XyShared &sh, cg::cluster_group &cl,
                               uint32_t &lo, uint32_t &hi, uint32_t &level, uint32_t phi,
                               uint32_t tlo, uint32_t thi, bool *finished) {
    XyShared *lead = cl.map_shared_rank(&sh, 0);
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
            if (k < hi) won = xy_expand<DIM>(p, __ldcg(p.list + k), phi, tlo, thi, nb);
            uint32_t pos = hi + warp_reserve(cnt, __popc(won));
#pragma unroll
            for (int s = 0; s < 2 * DIM; ++s) {
                if (won & (1u << s)) {
                    if (pos < p.g.N) p.list[pos] = nb.packed[s];
                    else raise_status(p.ctl, WOLFF_EINVAL, 0xF0u);
                    ++pos;
                }
            }
        }
        cl.sync();
        uint32_t added = *reinterpret_cast<volatile unsigned int *>(cnt);
        ++level;
        if (added > p.g.N - hi) {
            if (rank == 0 && threadIdx.x == 0) raise_status(p.ctl, WOLFF_EINVAL, 0xF1u);
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

// All CTAs: boundary sums over list[0, C), then reflect and release the
// members.  The leader's thread 0 gets the three sums.
template <int DIM>
__device__ void xy_team_finish(const StepParams &p, XyShared &sh, cg::cluster_group &cl,
                               uint32_t C, uint32_t phi, long long out[3]) {
    XyShared *lead = cl.map_shared_rank(&sh, 0);
    const unsigned int rank = cl.block_rank(), cs = cl.num_blocks();
    const uint32_t tid = rank * blockDim.x + threadIdx.x, nt = cs * blockDim.x;
    long long acc[3] = {0, 0, 0};
    for (uint32_t k = tid; k < C; k += nt) xy_boundary<DIM>(p, __ldcg(p.list + k), phi, acc);
    xy_block_sum3(sh, acc);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (acc[q] != 0) atomicAdd(&lead->sum[q], (unsigned long long)acc[q]);
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            out[q] = (long long)sh.sum[q];
            sh.sum[q] = 0;
        }
    }
    for (uint32_t k = tid; k < C; k += nt) {
        uint32_t c[DIM];
        unpack<DIM>(__ldcg(p.list + k), c);
        xy_flip(p, site_index<DIM>(p.g, c), phi);
        p.list[k] = kEmptySlot;
    }
    cl.sync();
}

template <int DIM>
__device__ void xy_worker(const StepParams &p, XyShared &sh, cg::cluster_group &cl) {
    XyShared *lead = cl.map_shared_rank(&sh, 0);
    while (true) {
        cl.sync();
        const volatile unsigned int *cmd = lead->cmd;
        const unsigned int kind = cmd[0];
        uint32_t lo = cmd[1], hi = cmd[2], level = cmd[3];
        const uint32_t phi = cmd[4], tlo = cmd[6], thi = cmd[7];
        if (kind == kXyLevels) {
            bool finished = false;
            xy_team_levels<DIM>(p, sh, cl, lo, hi, level, phi, tlo, thi, &finished);
        } else if (kind == kXyFinish) {
            long long out[3];
            xy_team_finish<DIM>(p, sh, cl, hi, phi, out);
        } else {
            cl.sync();   // the leader's shared memory outlives every remote read
            return;
        }
    }
}

__device__ __forceinline__ void xy_announce(XyShared &sh, cg::cluster_group &cl,
                                            unsigned int kind, uint32_t lo, uint32_t hi,
                                            uint32_t level, uint32_t phi, unsigned long long t) {
    if (threadIdx.x == 0) {
        sh.cmd[0] = kind;
        sh.cmd[1] = lo;
        sh.cmd[2] = hi;
        sh.cmd[3] = level;
        sh.cmd[4] = phi;
        sh.cmd[5] = 0;
        sh.cmd[6] = (uint32_t)t;
        sh.cmd[7] = (uint32_t)(t >> 32);
        sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
    }
    cl.sync();
}

template <int DIM>
__device__ void xy_leader(const StepParams &p, XyShared &sh, cg::cluster_group &cl) {
    DevCtl *ctl = p.ctl;
    uint32_t *w = reinterpret_cast<uint32_t *>(p.spins);
    const bool t0 = threadIdx.x == 0;
    const bool has_team = cl.num_blocks() > 1;
    const uint32_t nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long E = 0, Mx = 0, My = 0;
    unsigned long long total_C = 0;
    uint32_t last_C = 0, last_levels = 0;
    if (t0) {
        ctl->st_start_ns = global_ns();
        E = ctl->E;
        Mx = ctl->M;
        My = ctl->My;
        total_C = ctl->total_C;
        last_C = ctl->last_C;
        last_levels = ctl->last_levels;
        sh.sum[0] = sh.sum[1] = sh.sum[2] = 0;
    }
    for (unsigned long long u = 0; u < p.n; ++u) {
        const unsigned long long t = p.t0 + u;
        const uint32_t tlo = (uint32_t)t, thi = (uint32_t)(t >> 32);
        if (t0) {
            const Philox4 r = philox4x32_10(0u, tlo, thi, kTagSeed, p.key0, p.key1);
            const uint32_t i0 = (uint32_t)(((unsigned long long)r.v[0] * p.g.N) >> 32);
            atomicOr(w + i0, kXyMark);
            const uint32_t p0 = pack_index<DIM>(p.g, i0);
            p.list[0] = p0;
            sh.list[0] = p0;
            sh.front[0][0] = p0;
            sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0;
            sh.phi = (r.v[1] >> (32u - (p.xy_bits + 1u))) << (15u - p.xy_bits);
        }
        __syncthreads();
        const uint32_t phi = sh.phi;
        uint32_t C = 1, f = 1, level = 0, cur = 0;
        bool went_team = false;
        while (f > 0) {
            if (has_team && f > p.t_up) {
                went_team = true;
                xy_announce(sh, cl, kXyLevels, C - f, C, level, phi, t);
                uint32_t lo = C - f, hi = C;
                bool finished = false;
                xy_team_levels<DIM>(p, sh, cl, lo, hi, level, phi, tlo, thi, &finished);
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
                    won = xy_expand<DIM>(p, packed, phi, tlo, thi, nb);
                }
                uint32_t pos = warp_reserve(cnt, __popc(won));
#pragma unroll
                for (int s = 0; s < 2 * DIM; ++s) {
                    if (won & (1u << s)) {
                        const uint32_t gpos = C + pos;
                        if (gpos < p.g.N) p.list[gpos] = nb.packed[s];
                        else raise_status(ctl, WOLFF_EINVAL, 0xF3u);
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
        long long d[3] = {0, 0, 0};
        if (went_team || (has_team && C > kLocalListCap)) {
            xy_announce(sh, cl, kXyFinish, 0, C, level, phi, t);
            xy_team_finish<DIM>(p, sh, cl, C, phi, d);
        } else {
            const bool in_shared = C <= kLocalListCap;
            for (uint32_t k = threadIdx.x; k < C; k += blockDim.x)
                xy_boundary<DIM>(p, in_shared ? sh.list[k] : __ldcg(p.list + k), phi, d);
            xy_block_sum3(sh, d);
            __syncthreads();
            for (uint32_t k = threadIdx.x; k < C; k += blockDim.x) {
                uint32_t c[DIM];
                unpack<DIM>(in_shared ? sh.list[k] : __ldcg(p.list + k), c);
                xy_flip(p, site_index<DIM>(p.g, c), phi);
                p.list[k] = kEmptySlot;
            }
        }
        if (t0) {
            E += d[0];
            Mx += d[1];
            My += d[2];
            total_C += C;
            last_C = C;
            last_levels = level;
            if (p.xy_records) {
                wolff_xy_record r;
                r.C = C;
                r.levels = level;
                r.E = E;
                r.Mx = Mx;
                r.My = My;
                p.xy_records[u] = r;
            }
        }
        __syncthreads();
    }
    if (t0) {
        ctl->E = E;
        ctl->M = Mx;
        ctl->My = My;
        ctl->total_C = total_C;
        ctl->last_C = last_C;
        ctl->last_levels = last_levels;
        ctl->t = p.t0 + p.n;
        ctl->st_updates += p.n;
        ctl->st_end_ns = global_ns();
    }
    if (has_team) {
        xy_announce(sh, cl, kXyExit, 0, 0, 0, 0, 0);
        cl.sync();
    }
}

template <int DIM>
__global__ void __launch_bounds__(512, 1) k_xy_team(StepParams p) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ XyShared sh;
    if (cl.block_rank() != 0) {
        xy_worker<DIM>(p, sh, cl);
        return;
    }
    xy_leader<DIM>(p, sh, cl);
}

// Initial angles: the top `bits` bits of lane 0 of Philox(i, 0, 0, 2), on the grid.
__global__ void k_xy_init(uint32_t *w, uint32_t N, uint32_t bits, uint32_t k0, uint32_t k1) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const Philox4 r = philox4x32_10(i, 0u, 0u, kTagInit, k0, k1);
        w[i] = (r.v[0] >> (32u - bits)) << (16u - bits);
    }
}

// Full recount of E = sum_{i,d} I(theta_i - theta_nb(i,d)), Mx, My (rows along x).
template <int DIM>
__global__ void k_xy_measure(const uint32_t *w, Geometry g, const int32_t *tab, DevCtl *ctl) {
    const uint32_t rows = g.N / g.L;
    long long e = 0, mx = 0, my = 0;
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
            const uint32_t ti = w[base + x] & kXyAngle;
            const uint32_t xr = (x + 1 == g.L) ? 0 : x + 1;
            e += xy_cos(tab, ti + 65536u - (w[base + xr] & kXyAngle));
            e += xy_cos(tab, ti + 65536u - (w[yup + x] & kXyAngle));
            if (DIM == 3) e += xy_cos(tab, ti + 65536u - (w[zup + x] & kXyAngle));
            mx += xy_cos(tab, ti);
            my += xy_cos(tab, ti + 65536u - 16384u);
        }
    }
    e = block_sum(e);
    mx = block_sum(mx);
    my = block_sum(my);
    if (threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_E), (unsigned long long)e);
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_M), (unsigned long long)mx);
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->full_My), (unsigned long long)my);
    }
}

__global__ void k_xy_check(const uint32_t *w, uint32_t N, uint32_t bits, DevCtl *ctl) {
    const uint32_t off_grid = ((1u << (16u - bits)) - 1u) | ~kXyAngle;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        if (w[i] & off_grid) raise_status(ctl, WOLFF_EINVAL, i);
}

__global__ void k_xy_zero_full(DevCtl *ctl) {
    ctl->full_E = 0;
    ctl->full_M = 0;
    ctl->full_My = 0;
}

__global__ void k_xy_full_to_chain(DevCtl *ctl) {
    ctl->E = ctl->full_E;
    ctl->M = ctl->full_M;
    ctl->My = ctl->full_My;
}

unsigned xy_grid(unsigned long long work, unsigned long long cap) {
    unsigned long long b = work < cap ? work : cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_xy_init(uint32_t *words, Geometry g, uint32_t bits, uint32_t k0, uint32_t k1,
                           cudaStream_t s) {
    k_xy_init<<<xy_grid((g.N + 255) / 256, 4096), 256, 0, s>>>(words, g.N, bits, k0, k1);
    return cudaGetLastError();
}

cudaError_t launch_xy_measure(int dim, const uint32_t *words, Geometry g, const int32_t *tab,
                              DevCtl *ctl, int set_chain, cudaStream_t s) {
    k_xy_zero_full<<<1, 1, 0, s>>>(ctl);
    const unsigned blocks = xy_grid(g.N / g.L, 8192), threads = g.L >= 256 ? 256 : 64;
    if (dim == 2)
        k_xy_measure<2><<<blocks, threads, 0, s>>>(words, g, tab, ctl);
    else
        k_xy_measure<3><<<blocks, threads, 0, s>>>(words, g, tab, ctl);
    if (set_chain) k_xy_full_to_chain<<<1, 1, 0, s>>>(ctl);
    return cudaGetLastError();
}

cudaError_t launch_xy_check(const uint32_t *words, uint32_t N, uint32_t bits, DevCtl *ctl,
                            cudaStream_t s) {
    k_xy_check<<<xy_grid((N + 255) / 256, 4096), 256, 0, s>>>(words, N, bits, ctl);
    return cudaGetLastError();
}

cudaError_t launch_xy_team(int dim, const StepParams &p, int cluster_size, int threads,
                           cudaStream_t s) {
    const void *fn = dim == 2 ? reinterpret_cast<const void *>(&k_xy_team<2>)
                              : reinterpret_cast<const void *>(&k_xy_team<3>);
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
