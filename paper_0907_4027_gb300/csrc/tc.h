// tc.h -- host interface (internal to the library) of the separable GSW iteration on the
// tensor cores: tc.cu implements it, hot.cu drives it for contexts in HOT_PREC_TENSOR mode.
#pragma once
#include <cuda_runtime.h>

namespace hot_tc {

struct Plan;  // operand buffers, tensor maps and launch shapes of one context's traps

// One launch of a hot_gsw sequence, in the accumulator and weight buffers of the context.
struct Step {
  int M;
  const unsigned long long *acc_in;  // [2][M] sums of the previous forward (iterations)
  unsigned long long *acc_out;       // [2][M] zero on entry: sums of this launch's forward
  unsigned long long *acc_clear;     // [2][M] cleared for the launch after next
  const float *w_in;                 // [M] weights before the update
  float *w_out;                      // [M] weights after the update
  float *phi;                        // [H][W] phases: read (launch 0) or written (iterations)
  float *trace;                      // NULL, or e, u of the fields this launch reads
  float fx_scale, inv_fx_n;          // fixed-point scale 2^s of the sums; 1 / (N 2^s)
  int *err;                          // device flag set when a bounded wait runs out
  long long limit_ns;                // that bound
};

// Launch shapes of the tensor mode for a W x H hologram with M traps on `sms` SMs (host only).
struct Shape {
  int Kb, Kf;              // K of the back (2M) and forward (2W) GEMMs, padded to a K slice
  int rows_h;              // H padded to the tile height
  int bn_back, bn_fwd;     // tile widths (32, 64, 128 or 256)
  int rows_b, rows_f;      // 2W and 2M padded to the tile widths
  int fwd_splits, fwd_cps; // K splits of the forward GEMM and K slices per split
};
Shape shape_for(int W, int H, int M, int sms);

// Builds the operands of the traps' complex column and row tables Xc [M][W], Yc [M][H] (queued
// on st).  On failure returns the CUDA error and names the step in *what.
cudaError_t plan_create(Plan **out, int W, int H, int M, const float2 *Xc, const float2 *Yc, cudaStream_t st,
                        const char **what);
void plan_destroy(Plan *p);  // NULL-safe; the caller has synchronised the stream
// Rebuilds the operands after the tables changed in place (same M, W, H; 1 kernel).
cudaError_t plan_refresh(Plan *p, cudaStream_t st);

// Launch 0: the forward field of the phases s.phi (2 kernels).  pdl: the first kernel is a
// programmatic dependent of the previous kernel in the stream; chain: so are the others of
// their predecessors.
cudaError_t launch_forward(Plan *p, const Step &s, cudaStream_t st, bool pdl, bool chain, int *kernels);
// Launch k >= 1: weight update and coefficients, back-projection -> s.phi, forward field (3 kernels).
cudaError_t launch_iteration(Plan *p, const Step &s, cudaStream_t st, bool pdl, bool chain, int *kernels);

// C[rows][cols] = A[rows][K] B[cols][K]^T (device pointers, FP32) with the tensor-core GEMM of
// the iteration, operands split in two TF32 (operands = 0) or FP16 (operands = 1) parts, tile
// width tile_n (32, 64, 128 or 256); synchronous, allocates its operands.
cudaError_t gemm(int rows, int cols, int K, const float *A, const float *B, float *C, int tile_n, int operands,
                 cudaStream_t st, int *timed_out, const char **what);

}  // namespace hot_tc
