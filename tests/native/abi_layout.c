/* Prints the size and field offsets of every struct of the C ABI, for the
 * test that compares them with the Python binding's ctypes declarations. */
#include <stddef.h>
#include <stdio.h>

#include "hd.h"

#define F(T, m) printf(#T "." #m " %zu\n", offsetof(T, m))
#define S(T) printf(#T " %zu\n", sizeof(T))

int main(void) {
  S(hd_stream_info);
  F(hd_stream_info, nbits); F(hd_stream_info, nwords); F(hd_stream_info, nsub);
  S(hd_field);
  F(hd_field, words); F(hd_field, nwords); F(hd_field, nbits); F(hd_field, gap);
  F(hd_field, subseq_bits); F(hd_field, lengths); F(hd_field, alphabet); F(hd_field, n);
  S(hd_config);
  F(hd_config, subseq_bits); F(hd_config, threads); F(hd_config, window);
  F(hd_config, lut_bits); F(hd_config, cr_classes); F(hd_config, decoder);
  S(hd_serve_config);
  F(hd_serve_config, budget_bytes); F(hd_serve_config, slots); F(hd_serve_config, max_batch);
  F(hd_serve_config, queue_cap); F(hd_serve_config, direct);
  F(hd_serve_config, watchdog_us);
  S(hd_result);
  F(hd_result, status); F(hd_result, d_out); F(hd_result, n); F(hd_result, queue_us);
  F(hd_result, latency_us);
  S(hd_serve_stats_t);
  F(hd_serve_stats_t, timed_out_batches); F(hd_serve_stats_t, retired_batches);
  S(hd_lorenzo);
  F(hd_lorenzo, ndim); F(hd_lorenzo, radius); F(hd_lorenzo, dims); F(hd_lorenzo, eb);
  F(hd_lorenzo, out_idx); F(hd_lorenzo, out_val); F(hd_lorenzo, n_out);
  F(hd_lorenzo, chunk_slices); F(hd_lorenzo, band_rows); F(hd_lorenzo, separate);
  return 0;
}
