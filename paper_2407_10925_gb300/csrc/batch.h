// batch.h -- internal interface between the handle (lcs_bound.cu) and the
// batched persistent launch (batch.cu).
#pragma once

#include <vector>

#include <cuda_runtime.h>

#include "../../include/lcs_bound.h"
#include "lcs_common.h"

namespace lcs {

constexpr int kMaxBatch = 16;

struct BatchState;

lcs_status batch_create(int n, const int (*shapes)[3], const lcs_bound_opts& o, cudaStream_t s, BatchState** out);
lcs_status batch_iterate(BatchState* B, cudaStream_t s, long long n_iters);
lcs_status batch_report(BatchState* B, cudaStream_t s, int i, lcs_bound_report* out);
const long long* batch_vector(BatchState* B, cudaStream_t s, int i, int k, unsigned long long* n_stored,
                              unsigned long long* n_total, lcs_status* err);
lcs_status batch_set_spin_budget(BatchState* B, cudaStream_t s, long long cycles);
lcs_status batch_clear_status(BatchState* B, cudaStream_t s);
void batch_tuning(const BatchState* B, int* grid, int* units, double* ms, long long* launches, int* graph, int* mode,
                  double* ms_persistent, double* ms_concurrent, int* graph_captured, long long* graph_replays,
                  int* min_ctas_per_sm);
lcs_status batch_set_mode(BatchState* B, cudaStream_t s, int mode);
int batch_size(const BatchState* B);
int batch_d(const BatchState* B, int i);
void batch_destroy(BatchState* B);

// provided by lcs_bound.cu for the concurrent mode (the single-instance kernels)
// iter_base (may be null): a device count the kernel adds to iter
void launch_finalize_incr(const RedPartial* parts, int n, int r_mode, DevState* st, long long iter, cudaStream_t s,
                          const long long* iter_base = nullptr);
void launch_finalize_check(const RedPartial* parts, int n, DevState* st, long long iter, cudaStream_t s,
                           const long long* iter_base = nullptr);
int grid_for_work(const void* fn, int sms, unsigned long long work_items);

// provided by kernels_d2s.cu (d = 2, sigma >= 3, swap-aware)
int d2s_min_h(int sigma);
unsigned long long d2s_slots(int sigma, int h);
void launch_swap_check_d2s(int sigma, const long long* v, unsigned long long n, int h, DevState* st, int grid,
                           cudaStream_t s);

// provided by kernels_rt.cu: the general kernels (any d, full storage, f_mode 0)
const KernelSet* kernels_rt(int sigma);
// provided by kernels_s2d2.cu: the sigma = d = 2 swap-aware sweep over
// offset-normalised 32-bit storage
const KernelSet* kernels_s2d2_narrow();
// blocks: the block form (two phases, one thread per state in the second)
unsigned long long rt_work_items(int sigma, int d, unsigned long long n_states, unsigned long long n_tail, bool blocks);
// the block form of the general kernels: whether it serves (sigma, d, h), the
// length of its term-offset table, and the launch that fills the table
bool rt_blocks_apply(int sigma, int d, int h);
size_t rt_offsets_len(int sigma, int d);
void rt_offsets_fill(int sigma, int d, unsigned short* offs, unsigned* start, cudaStream_t s);
std::vector<unsigned long long> rt_tile_list(int sigma, int d, int h);

// provided by kernels_orbit.cu (sigma = d = 2 orbit form)
unsigned long long orbit_len(int h);
void launch_orbit_unpack(const long long* orb, long long* out, int h, unsigned long long n_tail, DevState* st,
                         cudaStream_t s);
void launch_orbit_pack(const long long* v, long long* orb, int h, unsigned long long n_tail, cudaStream_t s);

// provided by kernels_d3s.cu (sigma = 2, d = 3, permutation-aware)
int d3s_min_h();
int d3s_max_h();
unsigned long long d3s_tiles(int h);
void launch_perm_check_d3s(const long long* v, unsigned long long n_stored, unsigned long long n_total, DevState* st,
                           int grid, cudaStream_t s);

}  // namespace lcs
