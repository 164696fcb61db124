// wolff_capi.cu -- the C ABI declared in include/wolff.h.
//
// Host logic only: argument validation, the workspace layout, the bond
// threshold (computed here with the C library's exp so that the device never
// evaluates it), the choice of schedule and launch shape, checkpoint
// conversion and error latching.  All arithmetic of the update runs in the
// kernels of wolff_kernels.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "wolff.h"
#include "wolff_internal.h"
#include "wolff_tiny.h"

using namespace wolff;

namespace wolff {
cudaError_t launch_selftest_wait(DevCtl *scratch, unsigned long long wait_ns, cudaStream_t s);
}

struct wolff_ctx {
    int dim = 0, L = 0;
    uint32_t N = 0;
    int potts = 0;         // 0 = Ising, 1 = q-state Potts
    uint32_t q = 2;
    int xy = 0;            // 1 = XY model (32-bit site words)
    uint32_t angle_bits = 15;
    double xy_kk = 0;
    int32_t *xy_tab = nullptr;     // device copies in the workspace
    double *xy_coef = nullptr;
    std::vector<int32_t> h_xy_tab; // host copies (kept for the async uploads)
    std::vector<double> h_xy_coef;
    double J = 0, T = 0;
    uint64_t seed = 0, thr = 0;
    int layout = 0;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    DevCtl *ctl = nullptr;
    DevCtl *scratch_ctl = nullptr;
    uint8_t *spins = nullptr;
    uint32_t *list = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 0;
    int schedule = WOLFF_SCHED_CLUSTER;
    int blocks = 0, threads = 256;
    int tiny_threads = 256;        // CTA size of the tiny schedule
    int graph_blocks = 0, graph_threads = 0;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    uint64_t t_host = 0;
    void *rec_stage = nullptr;
    size_t rec_stage_bytes = 0;
    DevCtl *h_ctl = nullptr;       // pinned host copy of the control block (nullable)
    unsigned long long wait_ns = 2000000000ull;
    uint32_t t_up = 128, t_down = 64;
    bool thresholds_set = false;
    int win_levels = 0;   // window mode: growth levels per round (0 = off; set at init)
    uint8_t *ring = nullptr;      // pre-grown updates (lattices of kRingMinSites or more)
    int helpers_max = -1;         // helper teams: -1 = as many as fit, 0 = none, k = at most k
    int helpers_fit = -1;         // clusters that fit beside the main team (-1 = not asked yet)
    int helpers_fit_cluster = 0;  // ... for this cluster size and thread count
    int helpers_fit_threads = 0;
    uint32_t pg_epoch = 0;        // launches with helper teams so far
    int cluster = 8;
    int max_cluster = 8;
    std::string err;
};

namespace {

constexpr size_t kAlign = 256;
// window slots per CTA: one lattice per launch gets a 2048-update window at
// cluster size 16; the batched form keeps its CTAs small
constexpr int kPlainWindowSlots = 128;
constexpr int kBatchWindowSlots = 64;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool shape_ok(int dim, int L) {
    if (dim == 2) return L >= 2 && L <= 32767;
    if (dim == 3) return L >= 2 && L <= 1024;
    return false;
}

uint32_t sites(int dim, int L) {
    uint64_t n = 1;
    for (int d = 0; d < dim; ++d) n *= (uint64_t)L;
    return (uint32_t)n;
}

// AUTO's choice: the tiny schedule for Ising lattices of at most 64 words
// (2D L <= 32, 3D L <= 8), where warp 0 grows from registers and it was 9-29x
// faster than CLUSTER at 0.9-1.1 T_c from random and equilibrated starts;
// else CLUSTER.  On larger lattices TINY draws every site's bonds each update:
// 3-11x faster than CLUSTER while clusters are large (equilibrated at or
// below T_c) but up to 72x slower on clusters of a few sites, which window
// mode grows many at a time.
int auto_schedule(const wolff_ctx *c) {
    return (!c->potts && !c->xy && c->N <= WOLFF_TINY_MAX_SITES &&
            tiny_words_of(c->dim, c->L) <= 64u)
               ? WOLFF_SCHED_TINY
               : WOLFF_SCHED_CLUSTER;
}

wolff_status fail(wolff_ctx *c, wolff_status s, const char *msg) {
    if (c) c->err = msg;
    return s;
}

wolff_status cuda_fail(wolff_ctx *c, cudaError_t e, const char *where) {
    if (c) {
        c->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return WOLFF_ECUDA;
}

StepParams make_params(const wolff_ctx *c) {
    StepParams p;
    p.spins = c->spins;
    p.list = c->list;
    p.ctl = c->ctl;
    p.records = nullptr;
    p.g.L = (uint32_t)c->L;
    p.g.N = c->N;
    p.g.LL = (uint32_t)c->L * (uint32_t)c->L;
    p.key0 = (uint32_t)c->seed;
    p.key1 = (uint32_t)(c->seed >> 32);
    p.thr = c->thr;
    p.t0 = c->t_host;
    p.n = 0;
    p.wait_ns = c->wait_ns;
    p.t_up = c->t_up;
    p.t_down = c->t_down;
    p.win_levels = (uint32_t)c->win_levels;
    p.ring = c->ring;
    p.pg_epoch = c->pg_epoch;
    p.budget_ns = 0;
    p.q = c->q;
    p.xy_tab = c->xy_tab;
    p.xy_coef = c->xy_coef;
    p.xy_kk = c->xy_kk;
    p.xy_bits = c->angle_bits;
    p.xy_records = nullptr;
    return p;
}

// Synchronises and turns a latched device status into the return value.
wolff_status sync_and_check(wolff_ctx *c, DevCtl *host_copy) {
    DevCtl tmp;
    DevCtl *dst = host_copy ? host_copy : &tmp;
    // through the context's pinned copy when it has one (a direct DMA, no
    // staging through pageable memory)
    DevCtl *land = c->h_ctl ? c->h_ctl : dst;
    cudaError_t e = cudaMemcpyAsync(land, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronise");
    if (land != dst) memcpy(dst, land, sizeof(DevCtl));
    c->t_host = dst->t;   // the device's count (a time-budgeted run may stop early)
    if (dst->status != 0) {
        char buf[160];
        snprintf(buf, sizeof buf, "device reported %s (detail %u)",
                 wolff_status_string((wolff_status)dst->status), dst->err_detail);
        c->err = buf;
        return (wolff_status)dst->status;
    }
    return WOLFF_OK;
}

// Largest cluster size (16 or 8) the cluster schedule can launch here.
int max_cluster_size(int dim, int threads) {
    const void *fn = team_kernel(dim);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = window_smem_bytes(dim, threads, kPlainWindowSlots, 16);
    if (ensure_team_dyn_smem(dim, cfg.dynamicSmemBytes) != cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 8;
    }
    return 16;
}

// Every cluster-list slot holds kEmptySlot between updates.
cudaError_t empty_list(wolff_ctx *c) {
    return cudaMemsetAsync(c->list, 0xFF, (size_t)c->N * sizeof(uint32_t), c->stream);
}

// Device staging for host-bound records, kept by the context and grown on
// demand so that repeated calls do not allocate.
wolff_status ensure_rec_stage(wolff_ctx *c, size_t bytes) {
    if (bytes <= c->rec_stage_bytes) return WOLFF_OK;
    cudaStreamSynchronize(c->stream);
    if (c->rec_stage) cudaFree(c->rec_stage);
    c->rec_stage = nullptr;
    c->rec_stage_bytes = 0;
    if (cudaMalloc(&c->rec_stage, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, WOLFF_ENOMEM, "record staging buffer");
    }
    c->rec_stage_bytes = bytes;
    return WOLFF_OK;
}

// The Ising state transfers borrow the first N bytes of the cluster list as
// int8 scratch; this restores them (the rest of the list is untouched).
cudaError_t empty_scratch(wolff_ctx *c) {
    return cudaMemsetAsync(c->list, 0xFF, c->N, c->stream);
}

// Enqueues a bit-packed Ising lattice upload (ceil(N/32) words), the next
// update index and the recount; the words borrow the start of the list.
cudaError_t enqueue_ising_upload_bits(wolff_ctx *c, const uint32_t *h_bits, uint64_t t) {
    uint32_t *scratch = c->list;
    const size_t bytes = ((size_t)c->N + 31) / 32 * sizeof(uint32_t);
    const StepParams p = make_params(c);
    cudaError_t e = cudaMemcpyAsync(scratch, h_bits, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_reset_ctl(c->ctl, t, c->stream);
    if (e == cudaSuccess)
        e = launch_from_bits_measure(c->dim, c->spins, scratch, p.g, c->ctl, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0xFF, bytes, c->stream);
    if (e == cudaSuccess) c->t_host = t;
    return e;
}

// Enqueues a bit-packed download of the lattice into host memory.
cudaError_t enqueue_ising_download_bits(wolff_ctx *c, uint32_t *h_bits) {
    uint32_t *scratch = c->list;
    const size_t bytes = ((size_t)c->N + 31) / 32 * sizeof(uint32_t);
    cudaError_t e = launch_to_bits(scratch, c->spins, c->N, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_bits, scratch, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0xFF, bytes, c->stream);
    return e;
}

// Enqueues an Ising lattice upload (int8 +-1 from host memory), the next
// update index and the recount of E_bond and M; no synchronisation.
cudaError_t enqueue_ising_upload(wolff_ctx *c, const int8_t *h_spins, uint64_t t) {
    int8_t *scratch = reinterpret_cast<int8_t *>(c->list);
    const StepParams p = make_params(c);
    cudaError_t e = cudaMemcpyAsync(scratch, h_spins, c->N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_reset_ctl(c->ctl, t, c->stream);
    if (e == cudaSuccess)
        e = launch_from_pm1_measure(c->dim, c->spins, scratch, p.g, c->ctl, c->stream);
    if (e == cudaSuccess) e = empty_scratch(c);
    if (e == cudaSuccess) c->t_host = t;
    return e;
}

// Helper teams for a one-lattice cluster launch: the clusters that fit on the
// GPU beside the main team, while window mode is on and the lattice has a
// ring (and the launch's update count fits the helpers' 32-bit counters).
int plain_helpers(wolff_ctx *c, uint64_t n_updates) {
    if (!c->ring || c->potts || c->xy || c->win_levels == 0 || c->helpers_max == 0 ||
        n_updates < 2 || n_updates >= (1ull << 31))
        return 0;
    if (c->helpers_fit < 0 || c->helpers_fit_cluster != c->cluster ||
        c->helpers_fit_threads != c->threads) {
        const int fit = team_max_active_clusters(c->dim, c->cluster, c->threads, kPlainWindowSlots);
        c->helpers_fit = fit > 1 ? fit - 1 : 0;
        c->helpers_fit_cluster = c->cluster;
        c->helpers_fit_threads = c->threads;
    }
    int h = c->helpers_fit;
    if (c->helpers_max > 0 && h > c->helpers_max) h = c->helpers_max;
    return h;
}

// How far ahead of the main team's commits the helpers grow: the whole ring.
// Measured on the 10^4-update steps: a lead of the window plus a half or less
// leaves helpers behind the main team (more updates grown twice), the full
// ring was fastest in 2D and level in 3D.
uint32_t helper_lead(const wolff_ctx *) { return kRingSlots; }

// The main team's longest wait, at a launch's first window, for the helpers
// to grow it (they start with the launch): 20 us, about their time for one
// window's worth of updates.
constexpr unsigned long long kHelperFirstWaitNs = 20000ull;

int default_blocks(const wolff_ctx *c) {
    int b = (int)(c->N / 2048u);
    if (b < 1) b = 1;
    if (b > c->sm_count) b = c->sm_count;
    return b;
}

}  // namespace

extern "C" {

const char *wolff_status_string(wolff_status s) {
    switch (s) {
        case WOLFF_OK: return "WOLFF_OK";
        case WOLFF_EINVAL: return "WOLFF_EINVAL";
        case WOLFF_ENOMEM: return "WOLFF_ENOMEM";
        case WOLFF_ECUDA: return "WOLFF_ECUDA";
        case WOLFF_ETIMEOUT: return "WOLFF_ETIMEOUT";
        case WOLFF_EUNSUPPORTED: return "WOLFF_EUNSUPPORTED";
    }
    return "WOLFF_UNKNOWN";
}

uint64_t wolff_bond_threshold(double J, double T) {
    const double p = 1.0 - exp(-2.0 * J / T);
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return 1ull << 32;
    return (uint64_t)floor(ldexp(p, 32));
}

// The ring of pre-grown updates, on lattices large enough for helper teams.
static size_t ring_bytes(size_t n) {
    return n >= kRingMinSites ? (size_t)kRingSlots * kRingSlotBytes : 0;
}

size_t wolff_workspace_bytes(int dim, int L, int layout) {
    if (layout != WOLFF_LAYOUT_INT8 || !shape_ok(dim, L)) return 0;
    const size_t n = sites(dim, L);
    return 2 * sizeof(DevCtl) + round_up(n, kAlign) + round_up(n * sizeof(uint32_t), kAlign) +
           ring_bytes(n);
}

size_t wolff_xy_workspace_bytes(int dim, int L) {
    if (!shape_ok(dim, L)) return 0;
    const size_t n = sites(dim, L);
    return 2 * sizeof(DevCtl) + 2 * round_up(n * sizeof(uint32_t), kAlign) +
           round_up(kXyTableSize * sizeof(int32_t), kAlign) + round_up(17 * sizeof(double), kAlign);
}

static wolff_status init_common(wolff_ctx **out, int dim, int L, double J, double T,
                                uint64_t seed, int layout, void *d_workspace,
                                size_t workspace_bytes, void *stream, int potts, uint32_t q,
                                int xy_bits = 0);

wolff_status ising_init(wolff_ctx **out, int dim, int L, double J, double T, uint64_t seed,
                        int layout, void *d_workspace, size_t workspace_bytes, void *stream) {
    return init_common(out, dim, L, J, T, seed, layout, d_workspace, workspace_bytes, stream, 0, 2);
}

wolff_status potts_init(wolff_ctx **out, int dim, int L, int q, double J, double T, uint64_t seed,
                        void *d_workspace, size_t workspace_bytes, void *stream) {
    if (q < 2 || q > 64) return WOLFF_EINVAL;
    return init_common(out, dim, L, J, T, seed, WOLFF_LAYOUT_INT8, d_workspace, workspace_bytes,
                       stream, 1, (uint32_t)q);
}

wolff_status xy_init(wolff_ctx **out, int dim, int L, int angle_bits, double J, double T,
                     uint64_t seed, void *d_workspace, size_t workspace_bytes, void *stream) {
    if (!out) return WOLFF_EINVAL;
    *out = nullptr;
    if (angle_bits < 1 || angle_bits > WOLFF_XY_ANGLE_BITS) return WOLFF_EINVAL;
    return init_common(out, dim, L, J, T, seed, WOLFF_LAYOUT_INT8, d_workspace, workspace_bytes,
                       stream, 0, 2, angle_bits);
}

static wolff_status init_common(wolff_ctx **out, int dim, int L, double J, double T,
                                uint64_t seed, int layout, void *d_workspace,
                                size_t workspace_bytes, void *stream, int potts, uint32_t q,
                                int xy_bits) {
    if (!out) return WOLFF_EINVAL;
    *out = nullptr;
    if (!shape_ok(dim, L) || layout != WOLFF_LAYOUT_INT8) return WOLFF_EINVAL;
    if (!(J >= 0.0) || !(T > 0.0)) return WOLFF_EINVAL;
    const bool xy = xy_bits > 0;
    const size_t need = xy ? wolff_xy_workspace_bytes(dim, L) : wolff_workspace_bytes(dim, L, layout);
    if (d_workspace) {
        if (workspace_bytes < need) return WOLFF_ENOMEM;
        if (reinterpret_cast<uintptr_t>(d_workspace) % kAlign) return WOLFF_EINVAL;
    }
    wolff_ctx *c = new (std::nothrow) wolff_ctx;
    if (!c) return WOLFF_ENOMEM;
    c->dim = dim;
    c->win_levels = default_window_levels(dim);
    c->L = L;
    c->N = sites(dim, L);
    c->J = J;
    c->T = T;
    c->seed = seed;
    c->potts = potts;
    c->q = q;
    c->xy = xy ? 1 : 0;
    if (xy) {
        c->angle_bits = (uint32_t)xy_bits;
        c->xy_kk = ldexp(2.0 * J / T, -60);
        // round(cos(pi k / 32768) 2^30), k = 0..16384, and 1/n!, n = 0..16
        c->h_xy_tab.resize(kXyTableSize);
        for (uint32_t k = 0; k < kXyTableSize; ++k)
            c->h_xy_tab[k] = (int32_t)llround(cos(3.141592653589793 * (double)k / 32768.0) *
                                              1073741824.0);
        c->h_xy_coef.resize(17);
        c->h_xy_coef[0] = 1.0;
        for (int n = 1; n <= 16; ++n) c->h_xy_coef[n] = c->h_xy_coef[n - 1] / (double)n;
    }
    // Ising: p = 1 - exp(-2J/T); Potts: p = 1 - exp(-J/T)
    c->thr = potts ? wolff_bond_threshold(0.5 * J, T) : wolff_bond_threshold(J, T);
    c->layout = layout;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        delete c;
        return WOLFF_ECUDA;
    }
    if (d_workspace) {
        c->ws = d_workspace;
        c->ws_bytes = workspace_bytes;
    } else {
        if (cudaMalloc(&c->ws, need) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return WOLFF_ENOMEM;
        }
        c->own_ws = true;
        c->ws_bytes = need;
    }
    // pinned landing buffer for control-block reads (optional: without it
    // the reads stage through pageable memory)
    if (cudaMallocHost(reinterpret_cast<void **>(&c->h_ctl), sizeof(DevCtl)) != cudaSuccess) {
        cudaGetLastError();
        c->h_ctl = nullptr;
    }
    char *base = static_cast<char *>(c->ws);
    c->ctl = reinterpret_cast<DevCtl *>(base);
    c->scratch_ctl = reinterpret_cast<DevCtl *>(base + sizeof(DevCtl));
    c->spins = reinterpret_cast<uint8_t *>(base + 2 * sizeof(DevCtl));
    const size_t spin_bytes = round_up(xy ? (size_t)c->N * sizeof(uint32_t) : c->N, kAlign);
    c->list = reinterpret_cast<uint32_t *>(base + 2 * sizeof(DevCtl) + spin_bytes);
    if (!xy && ring_bytes(c->N))
        c->ring = reinterpret_cast<uint8_t *>(base + 2 * sizeof(DevCtl) + spin_bytes +
                                              round_up((size_t)c->N * sizeof(uint32_t), kAlign));
    if (xy) {
        char *tail = base + 2 * sizeof(DevCtl) + spin_bytes +
                     round_up((size_t)c->N * sizeof(uint32_t), kAlign);
        c->xy_tab = reinterpret_cast<int32_t *>(tail);
        c->xy_coef = reinterpret_cast<double *>(
            tail + round_up(kXyTableSize * sizeof(int32_t), kAlign));
    }
    c->blocks = default_blocks(c);
    c->threads = 512;
    c->max_cluster = max_cluster_size(dim, c->threads);
    c->cluster = c->max_cluster;
    if (auto_schedule(c) == WOLFF_SCHED_TINY) {
        c->schedule = WOLFF_SCHED_TINY;
        c->tiny_threads = tiny_default_threads(dim, L);
    }

    const StepParams p = make_params(c);
    e = cudaMemsetAsync(c->ws, 0, 2 * sizeof(DevCtl) + spin_bytes, c->stream);
    if (e == cudaSuccess) e = empty_list(c);
    // no ring entry may survive from whatever used this memory before (a
    // tag is unique only among this context's own launches)
    if (e == cudaSuccess && c->ring)
        e = cudaMemsetAsync(c->ring, 0, ring_bytes(c->N), c->stream);
    if (e == cudaSuccess) e = launch_reset_ctl(c->ctl, 0, c->stream);
    if (xy) {
        uint32_t *words = reinterpret_cast<uint32_t *>(c->spins);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->xy_tab, c->h_xy_tab.data(), kXyTableSize * sizeof(int32_t),
                                cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->xy_coef, c->h_xy_coef.data(), 17 * sizeof(double),
                                cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = launch_xy_init(words, p.g, c->angle_bits, p.key0, p.key1, c->stream);
        if (e == cudaSuccess)
            e = launch_xy_measure(dim, words, p.g, c->xy_tab, c->ctl, 1, c->stream);
    } else {
        if (e == cudaSuccess)
            e = potts ? launch_potts_init(c->spins, p.g, q, p.key0, p.key1, c->stream)
                      : launch_init(c->spins, p.g, p.key0, p.key1, c->stream);
        if (e == cudaSuccess)
            e = potts ? launch_potts_measure(dim, c->spins, p.g, c->ctl, 1, c->stream)
                      : launch_measure_full(dim, c->spins, p.g, c->ctl, 1, c->stream);
    }
    if (e != cudaSuccess) {
        cuda_fail(c, e, "ising_init");
        ising_free(c);
        return WOLFF_ECUDA;
    }
    wolff_status s = sync_and_check(c, nullptr);
    if (s != WOLFF_OK) {
        ising_free(c);
        return s;
    }
    *out = c;
    return WOLFF_OK;
}

wolff_status wolff_set_schedule(wolff_ctx *c, int schedule, int grid_blocks, int block_threads) {
    if (!c) return WOLFF_EINVAL;
    if (schedule < WOLFF_SCHED_AUTO || schedule > WOLFF_SCHED_TINY)
        return fail(c, WOLFF_EINVAL, "unknown schedule");
    if (schedule == WOLFF_SCHED_CLUSTER && grid_blocks != 0 && grid_blocks != 1 &&
        grid_blocks != 2 && grid_blocks != 4 && grid_blocks != 8 && grid_blocks != 16)
        return fail(c, WOLFF_EINVAL, "cluster size must be 1, 2, 4, 8 or 16");
    if (block_threads != 0 && (block_threads < 32 || block_threads > 1024 || block_threads % 32))
        return fail(c, WOLFF_EINVAL, "block_threads must be a multiple of 32 in [32, 1024]");
    if (grid_blocks < 0) return fail(c, WOLFF_EINVAL, "grid_blocks must be >= 0");
    // AUTO keeps to CLUSTER when the shape asked for is not a tiny one
    const bool tiny_shape = grid_blocks <= 1 &&
                            (block_threads == 0 || tiny_shape_ok(c->dim, c->L, block_threads));
    const int sched_eff = schedule != WOLFF_SCHED_AUTO ? schedule
                          : tiny_shape               ? auto_schedule(c)
                                                     : WOLFF_SCHED_CLUSTER;
    if (sched_eff == WOLFF_SCHED_TINY) {
        if (c->potts || c->xy)
            return fail(c, WOLFF_EUNSUPPORTED, "the tiny schedule runs the Ising update only");
        if (c->N > kTinyMaxSites)
            return fail(c, WOLFF_EUNSUPPORTED, "the tiny schedule takes at most 32768 sites");
        if (grid_blocks > 1) return fail(c, WOLFF_EINVAL, "the tiny schedule runs one CTA");
        const int thr = block_threads ? block_threads : tiny_default_threads(c->dim, c->L);
        if (!tiny_shape_ok(c->dim, c->L, thr))
            return fail(c, WOLFF_EINVAL,
                        "the tiny schedule needs a thread per two words of the lattice");
        c->schedule = WOLFF_SCHED_TINY;
        c->tiny_threads = thr;
        return WOLFF_OK;
    }
    if (c->potts && sched_eff != WOLFF_SCHED_CLUSTER)
        return fail(c, WOLFF_EUNSUPPORTED, "the Potts update runs on the cluster schedule only");
    if (c->xy && sched_eff != WOLFF_SCHED_CLUSTER)
        return fail(c, WOLFF_EUNSUPPORTED, "the XY update runs on the cluster schedule only");
    if (sched_eff != WOLFF_SCHED_GRAPH && (block_threads ? block_threads : c->threads) > 512)
        return fail(c, WOLFF_EINVAL, "persistent and cluster schedules take at most 512 threads");
    c->schedule = sched_eff;
    if (block_threads) c->threads = block_threads;
    if (c->schedule == WOLFF_SCHED_CLUSTER) {
        c->cluster = grid_blocks ? grid_blocks : c->max_cluster;
    } else {
        c->blocks = grid_blocks ? grid_blocks : default_blocks(c);
    }
    if (!c->thresholds_set) {   // measured defaults of each schedule
        c->t_up = c->schedule == WOLFF_SCHED_PERSISTENT ? 512u : 128u;
        c->t_down = c->t_up / 2;
    }
    if (c->gexec && (c->graph_blocks != c->blocks || c->graph_threads != c->threads)) {
        cudaGraphExecDestroy(c->gexec);
        cudaGraphDestroy(c->graph);
        c->gexec = nullptr;
        c->graph = nullptr;
    }
    return WOLFF_OK;
}

wolff_status wolff_set_local_thresholds(wolff_ctx *c, uint32_t t_up, uint32_t t_down) {
    if (!c) return WOLFF_EINVAL;
    if (t_up > kLocalFrontierCap || t_down > t_up)
        return fail(c, WOLFF_EINVAL, "need t_down <= t_up <= 2048");
    c->t_up = t_up;
    c->t_down = t_down;
    c->thresholds_set = true;
    return WOLFF_OK;
}

wolff_status wolff_set_burst(wolff_ctx *c, int enable) {
    if (!c) return WOLFF_EINVAL;
    if (enable < 0) return fail(c, WOLFF_EINVAL, "enable must be >= 0");
    c->win_levels = enable == 0 ? 0 : enable == 1 ? default_window_levels(c->dim)
                                                 : (enable > 64 ? 64 : enable);
    return WOLFF_OK;
}

wolff_status wolff_set_helpers(wolff_ctx *c, int max_helpers) {
    if (!c) return WOLFF_EINVAL;
    if (max_helpers < -1) return fail(c, WOLFF_EINVAL, "max_helpers must be >= -1");
    c->helpers_max = max_helpers;
    return WOLFF_OK;
}

wolff_status wolff_step(wolff_ctx *c, uint64_t n_updates, void *d_records) {
    if (!c) return WOLFF_EINVAL;
    if (n_updates == 0) return WOLFF_OK;
    StepParams p = make_params(c);
    p.records = reinterpret_cast<wolff_record *>(d_records);
    p.n = n_updates;
    cudaError_t e;
    // a large lattice may have been pushed out of L2 since the last call.  The
    // level-synchronous paths stream it back first; the Ising cluster path,
    // whose window mode touches scattered lines of tiny clusters, measured
    // faster without (the prefetch launch cost more than the misses it saved)
    const bool big = c->N >= (1u << 22);
    if (big && (c->potts || c->xy || c->schedule != WOLFF_SCHED_CLUSTER)) {
        e = launch_prefetch_l2(c->spins, (unsigned long long)c->N * (c->xy ? 4u : 1u), c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "prefetch");
    }
    if (c->xy) {
        StepParams px = p;
        px.records = nullptr;
        px.xy_records = reinterpret_cast<wolff_xy_record *>(d_records);
        e = launch_xy_team(c->dim, px, c->cluster, c->threads, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "xy launch");
    } else if (c->potts) {
        e = launch_potts_team(c->dim, p, c->cluster, c->threads, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "potts launch");
    } else if (c->schedule == WOLFF_SCHED_TINY) {
        e = launch_tiny(c->dim, p, nullptr, 1, c->L, c->tiny_threads, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "tiny launch");
    } else if (c->schedule == WOLFF_SCHED_CLUSTER) {
        const int helpers = plain_helpers(c, n_updates);
        StepParams ph = p;
        ph.pg_epoch = c->pg_epoch;
        ph.pg_lead = helper_lead(c);
        ph.pg_wait_ns = kHelperFirstWaitNs;
        e = launch_team(c->dim, ph, nullptr, 1, c->cluster, c->threads, kPlainWindowSlots,
                        c->stream, helpers);
        if (e != cudaSuccess) return cuda_fail(c, e, "cluster launch");
        if (helpers) ++c->pg_epoch;
    } else if (c->schedule == WOLFF_SCHED_GRAPH) {
        if (!c->gexec) {
            e = build_update_graph(c->dim, p, c->blocks, c->threads, &c->gexec, &c->graph);
            if (e != cudaSuccess) return cuda_fail(c, e, "build_update_graph");
            c->graph_blocks = c->blocks;
            c->graph_threads = c->threads;
        }
        e = launch_graph_call(c->ctl, n_updates, p.records, c->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(c->gexec, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    } else {
        int err = 0;
        const int per_sm = persistent_max_blocks_per_sm(c->dim, c->threads, &err);
        if (err) return cuda_fail(c, (cudaError_t)err, "occupancy");
        int blocks = c->blocks;
        if (blocks > per_sm * c->sm_count) blocks = per_sm * c->sm_count;
        if (blocks < 1) return fail(c, WOLFF_EUNSUPPORTED, "persistent kernel cannot be resident");
        void *args[] = {&p};
        e = launch_prelaunch(c->ctl, c->stream);
        if (e == cudaSuccess)
            e = cudaLaunchCooperativeKernel(persistent_kernel(c->dim), dim3(blocks),
                                            dim3(c->threads), args, 0, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "cooperative launch");
    }
    c->t_host += n_updates;
    return WOLFF_OK;
}

wolff_status measure(wolff_ctx *c, int64_t *E_bond, int64_t *M, uint64_t *last_C) {
    if (!c) return WOLFF_EINVAL;
    if (c->xy) return fail(c, WOLFF_EUNSUPPORTED, "XY contexts use xy_measure");
    DevCtl h;
    wolff_status s = sync_and_check(c, &h);
    if (s != WOLFF_OK) return s;
    if (E_bond) *E_bond = h.E;
    if (M) *M = h.M;
    if (last_C) *last_C = h.last_C;
    return WOLFF_OK;
}

wolff_status measure_full(wolff_ctx *c, int64_t *E_bond, int64_t *M) {
    if (!c) return WOLFF_EINVAL;
    if (c->xy) return fail(c, WOLFF_EUNSUPPORTED, "XY contexts use xy_measure_full");
    const StepParams p = make_params(c);
    cudaError_t e = c->potts ? launch_potts_measure(c->dim, c->spins, p.g, c->ctl, 0, c->stream)
                             : launch_measure_full(c->dim, c->spins, p.g, c->ctl, 0, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "measure_full");
    DevCtl h;
    wolff_status s = sync_and_check(c, &h);
    if (s != WOLFF_OK) return s;
    if (E_bond) *E_bond = h.full_E;
    if (M) *M = h.full_M;
    return WOLFF_OK;
}

wolff_status wolff_get_state(wolff_ctx *c, int8_t *h_spins, uint64_t *t) {
    if (!c) return WOLFF_EINVAL;
    if (c->xy) return fail(c, WOLFF_EUNSUPPORTED, "XY contexts use xy_get_state");
    if (h_spins && c->potts) {   // a Potts site's byte at rest is its colour
        cudaError_t e = cudaMemcpyAsync(h_spins, c->spins, c->N, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "get_state");
    } else if (h_spins) {
        int8_t *scratch = reinterpret_cast<int8_t *>(c->list);
        cudaError_t e = launch_to_pm1(scratch, c->spins, c->N, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_spins, scratch, c->N, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = empty_scratch(c);
        if (e != cudaSuccess) return cuda_fail(c, e, "get_state");
    }
    DevCtl h;
    wolff_status s = sync_and_check(c, &h);
    if (s != WOLFF_OK) return s;
    if (t) *t = h.t;
    return WOLFF_OK;
}

wolff_status wolff_set_state(wolff_ctx *c, const int8_t *h_spins, uint64_t t) {
    if (!c || !h_spins) return WOLFF_EINVAL;
    if (c->xy) return fail(c, WOLFF_EUNSUPPORTED, "XY contexts use xy_set_state");
    if (c->potts) {
        const StepParams p = make_params(c);
        cudaError_t e = cudaMemcpyAsync(c->spins, h_spins, c->N, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = launch_reset_ctl(c->ctl, t, c->stream);
        if (e == cudaSuccess) e = launch_potts_check(c->spins, c->N, c->q, c->ctl, c->stream);
        if (e == cudaSuccess) e = launch_potts_measure(c->dim, c->spins, p.g, c->ctl, 1, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "set_state");
        c->t_host = t;
        wolff_status st = sync_and_check(c, nullptr);
        if (st != WOLFF_OK) {   // leave a valid lattice behind a rejected one
            launch_potts_init(c->spins, p.g, c->q, p.key0, p.key1, c->stream);
            launch_reset_ctl(c->ctl, 0, c->stream);
            launch_potts_measure(c->dim, c->spins, p.g, c->ctl, 1, c->stream);
            cudaStreamSynchronize(c->stream);
            c->t_host = 0;
        }
        return st;
    }
    cudaError_t e = enqueue_ising_upload(c, h_spins, t);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_state");
    return sync_and_check(c, nullptr);
}

wolff_status wolff_run_host(wolff_ctx *c, const int8_t *h_spins_in, uint64_t t_in,
                            uint64_t n_updates, wolff_record *h_records, int8_t *h_spins_out) {
    if (!c) return WOLFF_EINVAL;
    if (c->xy) return fail(c, WOLFF_EUNSUPPORTED, "no host-buffer path for XY contexts");
    wolff_status s;
    if (h_spins_in) {
        // the upload is enqueued, not waited for: a rejected lattice (entries
        // other than +-1, read as -1) is reported by the one synchronisation
        // at the end of the call
        if (c->potts) {
            s = wolff_set_state(c, h_spins_in, t_in);
            if (s != WOLFF_OK) return s;
        } else {
            cudaError_t e = enqueue_ising_upload(c, h_spins_in, t_in);
            if (e != cudaSuccess) return cuda_fail(c, e, "upload");
        }
    }
    wolff_record *d_rec = nullptr;
    if (h_records && n_updates) {
        s = ensure_rec_stage(c, n_updates * sizeof(wolff_record));
        if (s != WOLFF_OK) return s;
        d_rec = reinterpret_cast<wolff_record *>(c->rec_stage);
    }
    s = wolff_step(c, n_updates, d_rec);
    if (s == WOLFF_OK && d_rec) {
        cudaError_t e = cudaMemcpyAsync(h_records, d_rec, n_updates * sizeof(wolff_record),
                                        cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) s = cuda_fail(c, e, "records copy");
    }
    if (s == WOLFF_OK && h_spins_out) {
        s = wolff_get_state(c, h_spins_out, nullptr);
    } else if (s == WOLFF_OK) {
        s = sync_and_check(c, nullptr);
    }
    return s;
}

wolff_status wolff_set_state_bits(wolff_ctx *c, const uint32_t *h_bits, uint64_t t) {
    if (!c || !h_bits) return WOLFF_EINVAL;
    if (c->potts || c->xy) return fail(c, WOLFF_EUNSUPPORTED, "bit-packed states are Ising only");
    cudaError_t e = enqueue_ising_upload_bits(c, h_bits, t);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_state_bits");
    return sync_and_check(c, nullptr);
}

wolff_status wolff_get_state_bits(wolff_ctx *c, uint32_t *h_bits, uint64_t *t) {
    if (!c) return WOLFF_EINVAL;
    if (c->potts || c->xy) return fail(c, WOLFF_EUNSUPPORTED, "bit-packed states are Ising only");
    if (h_bits) {
        cudaError_t e = enqueue_ising_download_bits(c, h_bits);
        if (e != cudaSuccess) return cuda_fail(c, e, "get_state_bits");
    }
    DevCtl h;
    wolff_status s = sync_and_check(c, &h);
    if (s != WOLFF_OK) return s;
    if (t) *t = h.t;
    return WOLFF_OK;
}

wolff_status wolff_run_host_bits(wolff_ctx *c, const uint32_t *h_bits_in, uint64_t t_in,
                                 uint64_t n_updates, wolff_record *h_records,
                                 uint32_t *h_bits_out) {
    if (!c) return WOLFF_EINVAL;
    if (c->potts || c->xy) return fail(c, WOLFF_EUNSUPPORTED, "bit-packed states are Ising only");
    if (h_bits_in) {
        cudaError_t e = enqueue_ising_upload_bits(c, h_bits_in, t_in);
        if (e != cudaSuccess) return cuda_fail(c, e, "upload");
    }
    wolff_record *d_rec = nullptr;
    if (h_records && n_updates) {
        wolff_status s = ensure_rec_stage(c, n_updates * sizeof(wolff_record));
        if (s != WOLFF_OK) return s;
        d_rec = reinterpret_cast<wolff_record *>(c->rec_stage);
    }
    wolff_status s = wolff_step(c, n_updates, d_rec);
    if (s == WOLFF_OK && d_rec) {
        cudaError_t e = cudaMemcpyAsync(h_records, d_rec, n_updates * sizeof(wolff_record),
                                        cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) s = cuda_fail(c, e, "records copy");
    }
    if (s == WOLFF_OK && h_bits_out) {
        cudaError_t e = enqueue_ising_download_bits(c, h_bits_out);
        if (e != cudaSuccess) s = cuda_fail(c, e, "download");
    }
    if (s == WOLFF_OK) s = sync_and_check(c, nullptr);
    return s;
}

wolff_status xy_measure(wolff_ctx *c, int64_t *E, int64_t *Mx, int64_t *My, uint64_t *last_C) {
    if (!c) return WOLFF_EINVAL;
    if (!c->xy) return fail(c, WOLFF_EUNSUPPORTED, "not an XY context");
    DevCtl h;
    wolff_status s = sync_and_check(c, &h);
    if (s != WOLFF_OK) return s;
    if (E) *E = h.E;
    if (Mx) *Mx = h.M;
    if (My) *My = h.My;
    if (last_C) *last_C = h.last_C;
    return WOLFF_OK;
}

wolff_status xy_measure_full(wolff_ctx *c, int64_t *E, int64_t *Mx, int64_t *My) {
    if (!c) return WOLFF_EINVAL;
    if (!c->xy) return fail(c, WOLFF_EUNSUPPORTED, "not an XY context");
    const StepParams p = make_params(c);
    cudaError_t e = launch_xy_measure(c->dim, reinterpret_cast<const uint32_t *>(c->spins), p.g,
                                      c->xy_tab, c->ctl, 0, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "xy_measure_full");
    DevCtl h;
    wolff_status s = sync_and_check(c, &h);
    if (s != WOLFF_OK) return s;
    if (E) *E = h.full_E;
    if (Mx) *Mx = h.full_M;
    if (My) *My = h.full_My;
    return WOLFF_OK;
}

wolff_status xy_get_state(wolff_ctx *c, uint16_t *h_theta, uint64_t *t) {
    if (!c) return WOLFF_EINVAL;
    if (!c->xy) return fail(c, WOLFF_EUNSUPPORTED, "not an XY context");
    if (h_theta) {
        // between updates a site word is its angle (no claim bit): copy the
        // low halves of the words, 2 bytes apart in a 4-byte stride
        cudaError_t e = cudaMemcpy2DAsync(h_theta, sizeof(uint16_t), c->spins, sizeof(uint32_t),
                                          sizeof(uint16_t), c->N, cudaMemcpyDeviceToHost,
                                          c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "xy_get_state");
    }
    DevCtl h;
    wolff_status s = sync_and_check(c, &h);
    if (s != WOLFF_OK) return s;
    if (t) *t = h.t;
    return WOLFF_OK;
}

wolff_status xy_set_state(wolff_ctx *c, const uint16_t *h_theta, uint64_t t) {
    if (!c || !h_theta) return WOLFF_EINVAL;
    if (!c->xy) return fail(c, WOLFF_EUNSUPPORTED, "not an XY context");
    const StepParams p = make_params(c);
    uint32_t *words = reinterpret_cast<uint32_t *>(c->spins);
    cudaError_t e = cudaMemsetAsync(words, 0, (size_t)c->N * sizeof(uint32_t), c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(words, sizeof(uint32_t), h_theta, sizeof(uint16_t),
                              sizeof(uint16_t), c->N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_reset_ctl(c->ctl, t, c->stream);
    if (e == cudaSuccess) e = launch_xy_check(words, c->N, c->angle_bits, c->ctl, c->stream);
    if (e == cudaSuccess) e = launch_xy_measure(c->dim, words, p.g, c->xy_tab, c->ctl, 1, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "xy_set_state");
    c->t_host = t;
    wolff_status st = sync_and_check(c, nullptr);
    if (st != WOLFF_OK) {   // leave a valid lattice behind a rejected one
        launch_xy_init(words, p.g, c->angle_bits, p.key0, p.key1, c->stream);
        launch_reset_ctl(c->ctl, 0, c->stream);
        launch_xy_measure(c->dim, words, p.g, c->xy_tab, c->ctl, 1, c->stream);
        cudaStreamSynchronize(c->stream);
        c->t_host = 0;
    }
    return st;
}

wolff_status wolff_get_info(wolff_ctx *c, wolff_info *info) {
    if (!c || !info) return WOLFF_EINVAL;
    info->dim = c->dim;
    info->L = c->L;
    info->N = c->N;
    info->thr = c->thr;
    info->seed = c->seed;
    info->t = c->t_host;
    info->schedule = c->schedule;
    info->grid_blocks = c->schedule == WOLFF_SCHED_CLUSTER ? c->cluster
                        : c->schedule == WOLFF_SCHED_TINY  ? 1
                                                           : c->blocks;
    info->block_threads = c->schedule == WOLFF_SCHED_TINY ? c->tiny_threads : c->threads;
    info->sm_count = c->sm_count;
    info->workspace_bytes = c->ws_bytes;
    info->helper_clusters = plain_helpers(c, 2);
    return WOLFF_OK;
}

wolff_status wolff_get_stats(wolff_ctx *c, wolff_stats *st) {
    if (!c || !st) return WOLFF_EINVAL;
    DevCtl h;
    wolff_status s = sync_and_check(c, &h);
    if (s != WOLFF_OK) return s;
    st->updates = h.st_updates;
    st->levels_local = h.st_levels_local;
    st->levels_grid = h.st_levels_grid;
    st->ns_local = h.st_ns_local;
    st->ns_grid = h.st_ns_grid;
    st->ns_finish = h.st_ns_finish;
    st->handoffs = h.st_handoffs;
    st->grid_finishes = h.st_grid_finishes;
    st->start_ns = h.st_start_ns;
    st->end_ns = h.st_end_ns;
    st->burst_updates = h.st_burst_updates;
    st->bursts = h.st_bursts;
    st->ns_win_grow = h.st_ns_win[0];
    st->ns_win_map = h.st_ns_win[1];
    st->ns_win_check = h.st_ns_win[2];
    st->ns_win_commit = h.st_ns_win[3];
    st->win_levels = h.st_win_levels;
    st->pregrown = h.st_pregrown;
    st->ns_win_first_grow = h.st_ns_win_first;
    st->win_regrown = h.st_win_regrown;
    st->win_fresh_grown = h.st_win_fresh_grown;
    return WOLFF_OK;
}

wolff_status wolff_philox(uint32_t key0, uint32_t key1, const uint32_t *d_ctr, uint32_t *d_out,
                          uint64_t n, void *stream) {
    if (n && (!d_ctr || !d_out)) return WOLFF_EINVAL;
    cudaError_t e = launch_philox(key0, key1, d_ctr, d_out, n, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? WOLFF_OK : WOLFF_ECUDA;
}

wolff_status ising_free(wolff_ctx *c) {
    if (!c) return WOLFF_OK;
    cudaStreamSynchronize(c->stream);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    if (c->rec_stage) cudaFree(c->rec_stage);
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    delete c;
    return WOLFF_OK;
}

const char *wolff_last_error(wolff_ctx *c) {
    if (!c) return "";
    return c->err.c_str();
}

struct wolff_batch {
    int capacity = 0;
    int win_slots = kBatchWindowSlots;   // window slots per CTA (0 = window mode off)
    int schedule = WOLFF_SCHED_CLUSTER;  // CLUSTER (teams) or TINY (one CTA per lattice)
    cudaStream_t stream = nullptr;
    StepParams *h_table = nullptr;   // pinned staging copy
    StepParams *d_table = nullptr;
    cudaEvent_t copied = nullptr;    // the staging copy may be overwritten after it
    bool pending = false;
};

wolff_status wolff_batch_create(wolff_batch **out, int capacity, void *stream) {
    if (!out || capacity <= 0 || capacity > (1 << 20)) return WOLFF_EINVAL;
    *out = nullptr;
    wolff_batch *b = new (std::nothrow) wolff_batch;
    if (!b) return WOLFF_ENOMEM;
    b->capacity = capacity;
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)capacity * sizeof(StepParams);
    if (cudaMallocHost(&b->h_table, bytes) != cudaSuccess ||
        cudaMalloc(&b->d_table, bytes) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        wolff_batch_free(b);
        return WOLFF_ENOMEM;
    }
    *out = b;
    return WOLFF_OK;
}

wolff_status wolff_batch_run(wolff_batch *b, wolff_ctx *const *ctxs, int n,
                             const uint64_t *n_updates, void *const *d_records, int cluster_size,
                             int block_threads) {
    return wolff_batch_run_timed(b, ctxs, n, n_updates, d_records, cluster_size, block_threads, 0);
}

wolff_status wolff_batch_run_timed(wolff_batch *b, wolff_ctx *const *ctxs, int n,
                                   const uint64_t *n_updates, void *const *d_records,
                                   int cluster_size, int block_threads, uint64_t budget_ns) {
    if (!b || n < 0 || n > b->capacity || (n && (!ctxs || !n_updates))) return WOLFF_EINVAL;
    const bool tiny = b->schedule == WOLFF_SCHED_TINY;
    if (cluster_size != 1 && (tiny || (cluster_size != 2 && cluster_size != 4 &&
                                       cluster_size != 8 && cluster_size != 16)))
        return WOLFF_EINVAL;
    if (tiny ? (block_threads != 0 && (block_threads < 32 || block_threads > 1024 ||
                                       block_threads % 32))
             : (block_threads < 32 || block_threads > 512 || block_threads % 32))
        return WOLFF_EINVAL;
    if (b->pending) {   // the previous staging copy must have been consumed
        if (cudaEventSynchronize(b->copied) != cudaSuccess) return WOLFF_ECUDA;
        b->pending = false;
    }
    // jobs: 2D first then 3D, each group largest lattice first
    int n2 = 0, n3 = 0;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return WOLFF_EINVAL;
        if (ctxs[i]->potts || ctxs[i]->xy) return WOLFF_EUNSUPPORTED;
        if (tiny && ctxs[i]->N > kTinyMaxSites) return WOLFF_EUNSUPPORTED;
        if (n_updates[i] == 0) continue;
        (ctxs[i]->dim == 2 ? n2 : n3) += 1;
    }
    int k2 = 0, k3 = n2;
    for (int i = 0; i < n; ++i) {
        wolff_ctx *c = ctxs[i];
        if (n_updates[i] == 0) continue;
        StepParams p = make_params(c);
        p.records = d_records ? reinterpret_cast<wolff_record *>(d_records[i]) : nullptr;
        p.n = n_updates[i];
        p.budget_ns = budget_ns;
        b->h_table[c->dim == 2 ? k2++ : k3++] = p;
    }
    auto by_size = [](const StepParams &a, const StepParams &c) { return a.g.N > c.g.N; };
    std::stable_sort(b->h_table, b->h_table + n2, by_size);
    std::stable_sort(b->h_table + n2, b->h_table + n2 + n3, by_size);
    const int total = n2 + n3;
    if (total == 0) return WOLFF_OK;
    cudaError_t e = cudaMemcpyAsync(b->d_table, b->h_table, (size_t)total * sizeof(StepParams),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->copied, b->stream);
    if (e != cudaSuccess) return WOLFF_ECUDA;
    b->pending = true;
    StepParams none = {};
    if (tiny) {
        // one CTA per lattice, one launch per dimension, shaped for the
        // largest lattice of that dimension (the table's first)
        for (int d = 2; d <= 3 && e == cudaSuccess; ++d) {
            const int cnt = d == 2 ? n2 : n3;
            if (!cnt) continue;
            const StepParams &first = b->h_table[d == 2 ? 0 : n2];
            const int maxL = (int)first.g.L;
            const int thr = block_threads ? block_threads : tiny_default_threads(d, maxL);
            if (!tiny_shape_ok(d, maxL, thr)) return WOLFF_EINVAL;
            e = launch_tiny(d, none, b->d_table + (d == 2 ? 0 : n2), cnt, maxL, thr, b->stream);
        }
    } else {
        if (n2)
            e = launch_team(2, none, b->d_table, n2, cluster_size, block_threads, b->win_slots,
                            b->stream);
        if (e == cudaSuccess && n3)
            e = launch_team(3, none, b->d_table + n2, n3, cluster_size, block_threads,
                            b->win_slots, b->stream);
    }
    if (e != cudaSuccess) return WOLFF_ECUDA;
    for (int i = 0; i < n; ++i) ctxs[i]->t_host += n_updates[i];
    return WOLFF_OK;
}

wolff_status wolff_batch_set_window(wolff_batch *b, int slots_per_cta) {
    if (!b) return WOLFF_EINVAL;
    if (slots_per_cta != 0 && slots_per_cta != 16 && slots_per_cta != 32 && slots_per_cta != 64 &&
        slots_per_cta != 128)
        return WOLFF_EINVAL;
    b->win_slots = slots_per_cta;
    return WOLFF_OK;
}

wolff_status wolff_batch_set_schedule(wolff_batch *b, int schedule) {
    if (!b) return WOLFF_EINVAL;
    if (schedule != WOLFF_SCHED_CLUSTER && schedule != WOLFF_SCHED_TINY) return WOLFF_EINVAL;
    b->schedule = schedule;
    return WOLFF_OK;
}

wolff_status wolff_batch_free(wolff_batch *b) {
    if (!b) return WOLFF_OK;
    if (b->copied) {
        cudaStreamSynchronize(b->stream);
        cudaEventDestroy(b->copied);
    }
    if (b->h_table) cudaFreeHost(b->h_table);
    if (b->d_table) cudaFree(b->d_table);
    delete b;
    return WOLFF_OK;
}

// Test hook for the failure-detection path: runs the library's bounded
// grid barrier on a private control block with two expected CTAs but only one
// launched, so the wait can only end by its time limit.  Writes the status
// the device latched (WOLFF_ETIMEOUT when the limit works) to *observed and
// leaves the context's own state untouched.
wolff_status wolff_selftest_wait_timeout(wolff_ctx *c, uint64_t wait_ns, int *observed) {
    if (!c || !observed) return WOLFF_EINVAL;
    if (wait_ns > 10000000000ull) return fail(c, WOLFF_EINVAL, "wait_ns above 10 s");
    cudaError_t e = cudaMemsetAsync(c->scratch_ctl, 0, sizeof(DevCtl), c->stream);
    if (e == cudaSuccess) e = launch_selftest_wait(c->scratch_ctl, wait_ns, c->stream);
    DevCtl h;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&h, c->scratch_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "selftest");
    *observed = (int)h.status;
    return WOLFF_OK;
}

}  // extern "C"
