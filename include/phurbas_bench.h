/*
 * phurbas_bench.h - measurement helper of libphurbas (not part of the method).
 *
 * phb_fma_peak runs a fixed, dependency-light chain of fused multiply-adds on
 * every SM so that the benchmark can measure the ALU peak that the fused fit
 * kernels are bounded by (the MLS accumulation is plain FP32 / FP64 FMA work,
 * not a tensor-core contraction).  precision: 0 = FP64, 1 = FP32.  Each of
 * blocks x 256 threads performs iters x 16 FMAs; `sink` (device, >= blocks*256
 * elements of the chosen type) receives the results so nothing is optimised
 * away.  Asynchronous on `stream`; returns 0, or 1 for invalid arguments, 3 on
 * a launch error.
 */
#ifndef PHURBAS_BENCH_H
#define PHURBAS_BENCH_H

#include <stdint.h>

#include "phurbas.h"

#ifdef __cplusplus
extern "C" {
#endif

int phb_fma_peak(int32_t precision, int32_t blocks, int32_t iters, void* sink, phb_stream_t stream);

/* Number of kernels this library has launched since load (host-side count,
 * incremented at every launch site). */
int64_t phb_launch_count(void);

/* Event trace of the fused fit and the neighbour search kernels.
 * phb_trace_start(capacity) creates `capacity` CUDA event pairs (timing
 * enabled) on the current device and arms the trace; every later launch of a
 * traced kernel records one pair around itself on its own stream, until the
 * pairs run out.  phb_trace_stop(ms, kernel_ids, capacity) synchronises on
 * the last recorded event, writes each launch's duration in milliseconds and
 * kernel id (1 = FP32-mixed fused fit, 2 = FP64 fused fit over all particles,
 * 3 = FP64 fit of the routed queue, 4 = neighbour search, 5 = list
 * compaction and tile plans, 6 and 7 = the tensor-core experiment's Gram and
 * solve kernels, 8 = corrected step of the FP32-mixed fits of refined tiles),
 * destroys the events and returns the number of
 * launches recorded (or -1 on a CUDA error).  Not thread-safe; one trace at a
 * time. */
int phb_trace_start(int32_t capacity);

/* Byte offset and size, inside the workspace, of the FP32 hi/lo records
 * written by every fit and step call (slot order, 24 floats per slot:
 * (xh, yh, zh, 0) (xl, yl, zl, 0) (rho, sigma, Vx, Vy)_h (..)_l
 * (Vz, Bx, By, Bz)_h (..)_l, with h = v rounded to FP32 and l = (v - h)
 * rounded to FP32), for tests that check them.  Host only.  Returns 0, or 1
 * for an invalid plan or NULL output. */
int phb_record_region(const phb_plan* plan, size_t* offset, size_t* bytes);

/* Copy diagnostic counters of the last operations on a workspace to the host
 * (synchronising on `stream`): out[0] = fits routed to FP64 by the last fused
 * fit, out[1] = tiles of the last neighbour build that read neighbours from
 * global memory (neighbourhood larger than the staging capacity), out[2] =
 * such tiles in the last fused fit, out[3] = number of tiles, out[4] = tiles
 * of the last FP32-mixed fused fit that took the corrected
 * semi-normal-equations step (phb_params.refine).  count <= 5.
 * Returns 0, 1 for invalid arguments, 3 on a CUDA error. */
int phb_workspace_stats(const phb_plan* plan, const void* ws, int32_t* out, int32_t count,
                        phb_stream_t stream);
int phb_trace_stop(float* ms, int32_t* kernel_ids, int32_t capacity);

/* Tensor-core experiment for the fit's accumulation (measurement only; no
 * other call uses it).  Same result as phb_mhd_rhs in FP32_MIXED with
 * refine = -1 and no FP64 routing, except that the moments and right-hand
 * sides of each particle are formed as the Gram matrix A^T W A of its
 * neighbour rows [p(q_j) | du_j] on the tensor cores: mma.sync m16n8k8 with
 * TF32 inputs split hi + lo (three products, FP32 accumulation), one warp per
 * particle in turn.  gram: device float [214][n] scratch (moments, right-hand
 * sides, neighbour count), gram_bytes >= 214 * 4 * n.  Trace ids 6 (Gram
 * kernel) and 7 (solve).  Needs plan->tile = 128 and the lists of the last
 * build; returns a phb_status. */
int phb_fit_tc_experiment(const phb_plan* plan, const phb_params* params, const double* pos,
                          const double* lambda, const double* U, void* ws, size_t ws_bytes,
                          float* gram, size_t gram_bytes, double* dudt, int32_t* status_word,
                          phb_stream_t stream);

/* Same read-out as phb_trace_stop without destroying the events or disarming
 * the trace.  For launches captured into a CUDA graph while the trace was
 * armed, the event pairs are recorded by the graph at every replay, so a read
 * after each replay gives that replay's kernel durations.  Returns the number
 * of recorded pairs (capped at capacity) or -1. */
int phb_trace_read(float* ms, int32_t* kernel_ids, int32_t capacity);

#ifdef __cplusplus
}
#endif

#endif
