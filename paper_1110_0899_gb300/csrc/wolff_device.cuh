// wolff_device.cuh -- device building blocks of the Wolff growth kernels.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), lattice coordinate
// packing, the idempotent atomic claim, warp-aggregated appends and the
// bounded grid-wide barrier that replaces the paper's quasi-block
// synchronisation (section 3).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wolff_internal.h"

namespace wolff {

constexpr unsigned kFullMask = 0xffffffffu;

// ---- Philox4x32-10 --------------------------------------------------------
// Round: multiply words 0 and 2 by the two round multipliers; the new words
// are (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)); the
// key advances by the Weyl increments between rounds.
struct Philox4 {
    uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1,
                                                 uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
    const uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
    const uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kMul0, c0);
        const uint32_t lo0 = kMul0 * c0;
        const uint32_t hi1 = __umulhi(kMul1, c2);
        const uint32_t lo1 = kMul1 * c2;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += kWeyl0;
        k1 += kWeyl1;
    }
    Philox4 out;
    out.v[0] = c0; out.v[1] = c1; out.v[2] = c2; out.v[3] = c3;
    return out;
}

// K independent Philox4x32-10 evaluations sharing the key and the last three
// counter words, run in lockstep so that their dependent multiply chains
// overlap (one evaluation's latency for all K).
template <int K>
__device__ __forceinline__ void philox4x32_10_lanes(const uint32_t c0[K], uint32_t c1,
                                                    uint32_t c2, uint32_t c3, uint32_t k0,
                                                    uint32_t k1, Philox4 out[K]) {
    const uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
    const uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
    uint32_t a[K], b[K], c[K], d[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        a[k] = c0[k];
        b[k] = c1;
        c[k] = c2;
        d[k] = c3;
    }
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint32_t hi0 = __umulhi(kMul0, a[k]);
            const uint32_t lo0 = kMul0 * a[k];
            const uint32_t hi1 = __umulhi(kMul1, c[k]);
            const uint32_t lo1 = kMul1 * c[k];
            a[k] = hi1 ^ b[k] ^ k0;
            b[k] = lo1;
            c[k] = hi0 ^ d[k] ^ k1;
            d[k] = lo0;
        }
        k0 += kWeyl0;
        k1 += kWeyl1;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        out[k].v[0] = a[k];
        out[k].v[1] = b[k];
        out[k].v[2] = c[k];
        out[k].v[3] = d[k];
    }
}

// ---- lattice coordinates ---------------------------------------------------
template <int DIM> struct Pack;
template <> struct Pack<2> {
    __host__ __device__ static constexpr int shift(int d) { return 16 * d; }
    static constexpr uint32_t kMask = 0xffffu;
};
template <> struct Pack<3> {
    __host__ __device__ static constexpr int shift(int d) { return 10 * d; }
    static constexpr uint32_t kMask = 0x3ffu;
};

template <int DIM>
__device__ __forceinline__ void unpack(uint32_t p, uint32_t c[DIM]) {
#pragma unroll
    for (int d = 0; d < DIM; ++d) c[d] = (p >> Pack<DIM>::shift(d)) & Pack<DIM>::kMask;
}

template <int DIM>
__device__ __forceinline__ uint32_t pack(const uint32_t c[DIM]) {
    uint32_t p = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) p |= c[d] << Pack<DIM>::shift(d);
    return p;
}

template <int DIM>
__device__ __forceinline__ uint32_t site_index(const Geometry &g, const uint32_t c[DIM]) {
    uint32_t i = c[0] + g.L * c[1];
    if (DIM == 3) i += g.LL * c[2];
    return i;
}

template <int DIM>
__device__ __forceinline__ uint32_t axis_stride(const Geometry &g, int d) {
    return d == 0 ? 1u : (d == 1 ? g.L : g.LL);
}

// Neighbours of a site: slot 2d = forward along axis d, slot 2d+1 = backward.
// Both the linear index and the packed coordinates are produced; unsigned
// wrap-around makes the +-(L-1) periodic jumps exact.
template <int DIM>
struct Neighbours {
    uint32_t idx[2 * DIM];
    uint32_t packed[2 * DIM];
};

template <int DIM>
__device__ __forceinline__ void neighbours(const Geometry &g, uint32_t p,
                                           uint32_t *self_idx,
                                           Neighbours<DIM> &nb) {
    uint32_t c[DIM];
    unpack<DIM>(p, c);
    const uint32_t i = site_index<DIM>(g, c);
    *self_idx = i;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const uint32_t cf = (c[d] + 1 == g.L) ? 0u : c[d] + 1;
        const uint32_t cb = (c[d] == 0) ? g.L - 1 : c[d] - 1;
        const uint32_t st = axis_stride<DIM>(g, d);
        nb.idx[2 * d] = i + (cf - c[d]) * st;
        nb.idx[2 * d + 1] = i + (cb - c[d]) * st;
        nb.packed[2 * d] = p + ((cf - c[d]) << Pack<DIM>::shift(d));
        nb.packed[2 * d + 1] = p + ((cb - c[d]) << Pack<DIM>::shift(d));
    }
}

// ---- claim -----------------------------------------------------------------
// Flips bit 0 of the site's byte from the seed spin to its opposite with one
// atomic on the containing 32-bit word: AND-clear when the seed spin is +1,
// OR-set when it is -1.  The operation is idempotent, so exactly one caller
// sees the old bit equal to the seed spin and wins the site.
__device__ __forceinline__ bool claim_site(uint8_t *spins, uint32_t j, uint32_t sig0bit) {
    unsigned int *w = reinterpret_cast<unsigned int *>(spins) + (j >> 2);
    const unsigned int bit = 1u << ((j & 3u) * 8u);
    if (sig0bit) {
        const unsigned int old = atomicAnd(w, ~bit);
        return (old & bit) != 0u;
    }
    const unsigned int old = atomicOr(w, bit);
    return (old & bit) == 0u;
}

// ---- small PTX helpers -----------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long atom_add_acq_rel_u64(unsigned long long *p,
                                                                   unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;"
                 : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// A spin byte read while another team of the launch may be writing it (the
// pre-growing helpers read the lattice the main team commits to): relaxed
// accesses at GPU scope, so each read returns a value some write stored.
__device__ __forceinline__ uint32_t ld_relaxed_u8(const uint8_t *p) {
    unsigned short v;
    asm volatile("ld.relaxed.gpu.global.u8 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_relaxed_u8(uint8_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u8 [%0], %1;" ::"l"(p), "h"((unsigned short)v)
                 : "memory");
}

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int *p) {
    return *reinterpret_cast<const volatile unsigned int *>(p);
}

__device__ __forceinline__ void raise_status(DevCtl *ctl, unsigned int code,
                                             unsigned int detail) {
    if (atomicCAS(&ctl->status, 0u, code) == 0u) ctl->err_detail = detail;
}

// ---- bounded waits -----------------------------------------------------------
// Polls *word until it differs from `seen`.  Gives up after wait_ns
// nanoseconds (globaltimer) without progress or 2^28 polls, or as soon as
// another CTA has raised an error.  `progress` (nullable) is a word whose
// change counts as progress and restarts the clock (a worker waiting for the
// next command while the leader completes updates on its own).  Returns the
// new value, or `seen` after raising WOLFF_ETIMEOUT / seeing an error.
__device__ __forceinline__ unsigned int bounded_wait_change(DevCtl *ctl, const unsigned int *word,
                                                            unsigned int seen,
                                                            const unsigned long long *progress,
                                                            unsigned long long wait_ns,
                                                            unsigned int where, bool *ok) {
    unsigned long long start = global_ns();
    unsigned long long last_progress = progress ? *(const volatile unsigned long long *)progress : 0;
    unsigned int polls = 0;
    *ok = true;
    while (true) {
        const unsigned int v = ld_acquire_u32(word);
        if (v != seen) return v;
        if ((++polls & 63u) == 0u) {
            if (ld_volatile_u32(&ctl->status) != 0u) { *ok = false; return seen; }
            const unsigned long long now = global_ns();
            if (progress) {
                const unsigned long long pv = *(const volatile unsigned long long *)progress;
                if (pv != last_progress) { last_progress = pv; start = now; }
            }
            if (now - start > wait_ns || polls > (1u << 28)) {
                raise_status(ctl, WOLFF_ETIMEOUT, where);
                *ok = false;
                return seen;
            }
        }
    }
}

// ---- bounded team barrier that carries the append count ---------------------
// bar_word = arrivals << 32 | entries appended since the team's phase began.
// The warps reserve cluster-list slots by adding to the low half during a
// level and every CTA arrives by adding 2^32, so the CTA whose add makes the
// arrivals reach (phase+1)*nblocks is the last one and reads the appended
// total from the same atomic.  It publishes (generation+1, total) in bar_pub;
// the others poll bar_pub (bounded: wait_ns of globaltimer without change or
// 2^28 polls raise WOLFF_ETIMEOUT; an error raised elsewhere also ends the
// wait).  The word is reset only when a new phase is published, while every
// other CTA is idle, so no reset can race with a reservation.
//   full = false: relaxed arrival and publication.  Enough between growth
//     levels: claims are atomics already performed when a CTA arrives, and
//     list entries are recognised by the empty-slot sentinel.
//   full = true: acq_rel arrival, release publication, acquire polling.
//     Needed where plain stores or reductions must be visible after the
//     barrier (the unmark pass).
// Returns false if the wait failed; the caller must leave the kernel.
// `gen` and `phase` are the CTA's copies (meaningful in thread 0).
__device__ __forceinline__ bool team_barrier(DevCtl *ctl, unsigned int nblocks, unsigned int &gen,
                                             unsigned int &phase, bool full,
                                             unsigned long long wait_ns, unsigned int where,
                                             unsigned int *count) {
    __shared__ unsigned int s_ok, s_val;
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = true;
        const unsigned int my = gen;
        unsigned int val = 0;
        const unsigned int last = (phase + 1u) * nblocks - 1u;
        const unsigned long long old = full ? atom_add_acq_rel_u64(&ctl->bar_word, 1ull << 32)
                                            : atomicAdd(&ctl->bar_word, 1ull << 32);
        if ((unsigned int)(old >> 32) == last) {
            val = (unsigned int)old;
            const unsigned long long pub = ((unsigned long long)(my + 1) << 32) | val;
            if (full) st_release_u64(&ctl->bar_pub, pub);
            else st_relaxed_u64(&ctl->bar_pub, pub);
        } else {
            unsigned long long start = global_ns();
            unsigned int polls = 0;
            while (true) {
                const unsigned long long v = full ? ld_acquire_u64(&ctl->bar_pub)
                                                  : ld_relaxed_u64(&ctl->bar_pub);
                if ((unsigned int)(v >> 32) != my) { val = (unsigned int)v; break; }
                if ((++polls & 63u) == 0u) {
                    if (ld_volatile_u32(&ctl->status) != 0u) { ok = false; break; }
                    if (global_ns() - start > wait_ns || polls > (1u << 28)) {
                        raise_status(ctl, WOLFF_ETIMEOUT, where);
                        ok = false;
                        break;
                    }
                }
            }
        }
        gen = my + 1;
        phase += 1;
        if (ld_volatile_u32(&ctl->status) != 0u) ok = false;
        s_val = val;
        s_ok = ok ? 1u : 0u;
    }
    __syncthreads();
    if (count) *count = s_val;
    return s_ok != 0u;
}

// Waits until list slot k holds this update's entry (bounded like the
// barrier).  Returns kEmptySlot if the wait failed; the status word then says
// why and the caller's next barrier ends the kernel.
__device__ __forceinline__ uint32_t wait_slot(const StepParams &p, uint32_t k) {
    uint32_t v = __ldcg(p.list + k);
    if (v != kEmptySlot) return v;
    const unsigned long long start = global_ns();
    unsigned int polls = 0;
    while (true) {
        v = ld_volatile_u32(p.list + k);
        if (v != kEmptySlot) return v;
        if ((++polls & 31u) == 0u) {
            if (ld_volatile_u32(&p.ctl->status) != 0u) return kEmptySlot;
            if (global_ns() - start > p.wait_ns || polls > (1u << 26)) {
                raise_status(p.ctl, WOLFF_ETIMEOUT, 6);
                return kEmptySlot;
            }
        }
    }
}

// Unmark: bit 1 of a member takes the member's new spin (= its bit 0), with a
// reduction on the containing word so that it never races a later claim of a
// neighbouring byte.
__device__ __forceinline__ void unmark_site(uint8_t *spins, uint32_t j, uint32_t sig0bit) {
    unsigned int *w = reinterpret_cast<unsigned int *>(spins) + (j >> 2);
    const unsigned int bit1 = 2u << ((j & 3u) * 8u);
    if (sig0bit) atomicAnd(w, ~bit1);
    else atomicOr(w, bit1);
}

// ---- warp-aggregated append -------------------------------------------------
// Each lane contributes `mine` entries; one atomicAdd per warp reserves the
// warp's range in the cluster list.  Returns the lane's first slot.  All 32
// lanes must call it.
// The counter is a 32-bit word (shared or global) or the 64-bit barrier word,
// whose low half counts entries.
__device__ __forceinline__ uint32_t reserve_add(unsigned int *c, uint32_t n) {
    return atomicAdd(c, n);
}
__device__ __forceinline__ uint32_t reserve_add(unsigned long long *c, uint32_t n) {
    return (uint32_t)atomicAdd(c, (unsigned long long)n);
}

template <typename Counter>
__device__ __forceinline__ uint32_t warp_reserve(Counter *counter, uint32_t mine) {
    const int lane = threadIdx.x & 31;
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullMask, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(kFullMask, incl, 31);
    uint32_t base = 0;
    if (total != 0u) {
        if (lane == 31) base = reserve_add(counter, total);
        base = __shfl_sync(kFullMask, base, 31);
    }
    return base + incl - mine;
}

// ---- block reduction of a 64-bit sum ---------------------------------------
__device__ __forceinline__ long long block_sum(long long v) {
    __shared__ long long s_part[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFullMask, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) s_part[warp] = v;
    __syncthreads();
    long long total = 0;
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        total = lane < nw ? s_part[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) total += __shfl_down_sync(kFullMask, total, o);
    }
    return total;   // valid in thread 0
}

// ---- the expansion of one wave-front site (step (iii') of section 4) -------
// Issues the 2*DIM neighbour loads (L2, bypassing L1 because other CTAs
// write them) and, while they are in flight, the DIM+1 Philox draws the
// site's bonds need -- its own call for the forward bonds, each backward
// neighbour's call for the bond it owns -- interleaved so that they cost one
// draw's latency.  Then claims only the neighbours still parallel to the seed
// spin behind an active bond: atomics from one thread overlap poorly, so
// they are spent only where a claim can succeed.  Returns the mask of
// neighbour slots won; nb receives their coordinates.
template <int DIM>
__device__ __forceinline__ uint32_t expand_site(const StepParams &p, uint32_t packed,
                                                uint32_t sig0bit, uint32_t tlo,
                                                uint32_t thi, Neighbours<DIM> &nb) {
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
    // decide every claim first, then issue the atomics back to back: a claim
    // whose outcome gated the next one would serialise their latencies
    uint32_t want = 0;
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) {
        const int d = s >> 1;
        const uint32_t r = (s & 1) ? draw[d + 1].v[d] : draw[0].v[d];
        if ((uint32_t)(v[s] & 1u) == sig0bit && (unsigned long long)r < p.thr) want |= 1u << s;
    }
    unsigned int old[2 * DIM];
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) {
        old[s] = 0;
        if (want & (1u << s)) {
            unsigned int *w = reinterpret_cast<unsigned int *>(p.spins) + (nb.idx[s] >> 2);
            const unsigned int bit = 1u << ((nb.idx[s] & 3u) * 8u);
            old[s] = sig0bit ? atomicAnd(w, ~bit) : atomicOr(w, bit);
        }
    }
    uint32_t won = 0;
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) {
        const unsigned int bit = 1u << ((nb.idx[s] & 3u) * 8u);
        // the claim wins when bit 0 still held the seed spin (see claim_site)
        if ((want & (1u << s)) && (((old[s] & bit) != 0u) == (sig0bit != 0u))) won |= 1u << s;
    }
    return won;
}

// Boundary term of one member: for every neighbour outside the cluster,
// +1 if it is anti-parallel to the seed spin (the bond gains energy when the
// member flips) and -1 if it is parallel; members have differing bits.
template <int DIM>
__device__ __forceinline__ int boundary_term(const StepParams &p, uint32_t packed,
                                             uint32_t sig0bit, uint32_t *self_idx) {
    Neighbours<DIM> nb;
    neighbours<DIM>(p.g, packed, self_idx, nb);
    int acc = 0;
#pragma unroll
    for (int s = 0; s < 2 * DIM; ++s) {
        const uint32_t v = __ldcg(p.spins + nb.idx[s]);
        const uint32_t cur = v & 1u, orig = (v >> 1) & 1u;
        if (cur == orig) acc += (orig == sig0bit) ? -1 : 1;
    }
    return acc;
}

// Seed site of update t: floor(x * N / 2^32), x = lane 0 of the seed draw.
__device__ __forceinline__ uint32_t seed_site(const StepParams &p, unsigned long long t) {
    const Philox4 r = philox4x32_10(0u, (uint32_t)t, (uint32_t)(t >> 32), kTagSeed,
                                    p.key0, p.key1);
    return (uint32_t)(((unsigned long long)r.v[0] * p.g.N) >> 32);
}

template <int DIM>
__device__ __forceinline__ uint32_t pack_index(const Geometry &g, uint32_t i) {
    uint32_t c[DIM];
    c[0] = i % g.L;
    if (DIM == 2) {
        c[1] = i / g.L;
    } else {
        c[1] = (i / g.L) % g.L;
        c[DIM - 1] = i / g.LL;
    }
    return pack<DIM>(c);
}

}  // namespace wolff
