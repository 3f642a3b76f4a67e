// Host-side launch wrappers of the libeprop kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace eprop {

struct Net;
struct GridBar;

void launch_inject(const Net &n, int i, int max_events_per_step, cudaStream_t st);
void launch_neuron(const Net &n, int i, int sm_count, cudaStream_t st);
void launch_readout(const Net &n, int i, int sm_count, cudaStream_t st);
void launch_deliver(const Net &n, int i, int grid_x, cudaStream_t st);

void prepare_kernel_attributes();
void prepare_step_kernel_attributes();
void launch_begin_call(const Net &n, int continuous, cudaStream_t st);
void launch_end_call(const Net &n, int T, cudaStream_t st);
void launch_filter_error(const Net &n, int i_end, cudaStream_t st);
int launch_tables(const Net &n, int i_end, cudaStream_t st);
void launch_trace_window(const Net &n, int i_end, int grid_x, cudaStream_t st);
// dense window update of a batch (batch > 1 with update windows), one
// state per sample and synapse
constexpr int kBatchWindowMax = 64;
void launch_window_batched(const Net &n, int i_end, int sm_count, cudaStream_t st);
void launch_trace_batched(const Net &n, int sm_count, cudaStream_t st);
void launch_window_pass(const Net &n, int i_end, int grid_x, int grid_idle, cudaStream_t st);
void launch_pred_input(const Net &n, int i, cudaStream_t st);
void launch_pred_apply(const Net &n, int i, cudaStream_t st);
void launch_readout_weights(const Net &n, int i_end, cudaStream_t st);
void launch_rollover(const Net &n, int i_end, cudaStream_t st);
void launch_flush(const Net &n, int i_end, float *w_dst, float *g_dst, long long q_begin, long long q_end,
                  int write_back, int sm_count, cudaStream_t st);
void launch_fill_int(int *p, long long count, int value, cudaStream_t st);
void launch_unpack_raster(const Net &n, unsigned char *dst, cudaStream_t st);
void launch_adam(const Net &n, int sm_count, cudaStream_t st);
int persistent_blocks(int sm_count);
cudaError_t launch_persistent_steps(const Net &n, int T, GridBar *gb, int blocks, cudaStream_t st);
void prepare_learning_signal_attributes();
// band-major learning state (trace_kernel 4)
int band_width(bool alif);
size_t band_window_smem(const Net &n);
int band_stages_fit(bool alif, int rr_stride);
uint32_t band_stage_size(bool alif, int rr_stride);
void launch_band_count(const long long *row_ptr, const uint32_t *tgt_d, int S, int W, int nb, int *seg);
void launch_band_chunk_sum(const int *seg, int S, int nb, int chunk, long long *part);
void launch_band_chunk_scan(int *seg, int S, int nb, int chunk, const long long *off);
void launch_band_tiles(const int *seg, const long long *band_tile0, int S, int nb, long long n_tiles, int4 *tiles,
                       unsigned *flag);
void launch_band_scatter(const Net &n, const float *w_src, uint32_t *bd_td, float *w_b);
void launch_band_gather(const Net &n, int r0, int r1, long long q_begin, float *w_dst, float *g_dst,
                        cudaStream_t st);
void launch_window_band(const Net &n, int i_end, int sm_count, cudaStream_t st);
void launch_deliver_band(const Net &n, int i, int grid_x, cudaStream_t st);
void prepare_band_attributes();
void launch_learning_signals(const float *fb, const float *E, float *L, int N, int U, int K, int B,
                             unsigned *err, cudaStream_t st);

}  // namespace eprop
