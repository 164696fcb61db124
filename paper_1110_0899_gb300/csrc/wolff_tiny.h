// wolff_tiny.h -- the tiny schedule's launch interface (wolff_tiny.cu), used
// by the C ABI.  One CTA per job holds the whole lattice in shared memory as
// bit planes (rows of ceil(L/32) 32-bit words); jobs come from d_table
// (njobs entries of side at most max_L) or the single job.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "wolff_internal.h"

namespace wolff {

constexpr uint32_t kTinyMaxSites = WOLFF_TINY_MAX_SITES;
uint32_t tiny_words_of(int dim, int L);            // (N / L) ceil(L / 32)
// warp 0 alone grows (64 or more threads, at most 64 words)
bool tiny_warp_mode(int dim, int L, int threads);
// a CTA of `threads` threads can run the lattice (each grower owns <= 2 words)
bool tiny_shape_ok(int dim, int L, int threads);
size_t tiny_smem_bytes(int dim, int L);
// the CTA size the tiny schedule takes by default for this lattice
int tiny_default_threads(int dim, int L);
cudaError_t launch_tiny(int dim, const StepParams &single, const StepParams *d_table, int njobs,
                        int max_L, int threads, cudaStream_t s);

}  // namespace wolff
