// gsw_kernels.cuh -- sm_103a kernels of the GSW hologram engine.
//
// Hot path (Sec. 3-4 of Bianchi & Di Leonardo): per iteration one kernel does the weight
// update of iteration k (Sec. 3), the back-projection phi_j = arg sum_m c_m e^{i Delta_j^m}
// and the forward field of iteration k+1 (Eq. 1).  Every sub-tile adds its per-trap sums of
// e^{i (phi_j - Delta_j^m)} into 64-bit fixed-point accumulators with integer atomics, which
// are exact and therefore independent of the order in which blocks arrive.  The next launch
// reads the completed sums: every block forms V_m, <|V|>, the new weights and the
// coefficients c_m = w_m V_m/|V_m| itself, in the same fixed order, so no block waits for
// another and no reduction tail sits between iterations.  Accumulators rotate over three
// buffers (read, written, cleared) and weights over two.  No FP64 runs per iteration.
//
// Per pair the kernels take exactly one complex exponential and accumulate it without a
// complex multiply: the back-projection folds the phase of its coefficient into the argument,
// S_j += w_m e^{i (Delta_j^m + arg V_m)}, and the forward field evaluates Eq. 1 as written,
// V_m += e^{i (phi_j - Delta_j^m)} (the fast mode with a per-sub-tile rotation of the phases
// that it undoes on each sub-tile's sums: see forward_traps).
//
// Phase generation: Eq. 2 splits into a column part and a row part,
//   Delta_j^m / 2pi = [a_m ix' + c_m ix'^2] + [b_m iy' + c_m iy'^2]
// with a_m = x_m p/(lambda f), b_m = y_m p/(lambda f), c_m = z_m p^2/(2 lambda f^2),
// ix' = ix - floor(W/2), iy' = iy - floor(H/2).  Each bracket is reduced modulo one turn
// in FP64 once per (trap, column) and (trap, row) when the traps are set, and stored as
// FP32.  Per (pixel, trap) pair the kernels add the two reduced parts (one FADD) and take
// one complex exponential: sin.approx/cos.approx on the SFU (fast) or sincospif
// (accurate).  Delta itself is never stored.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hot {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kTileW = 32;      // pixels per sub-tile row: one per lane
constexpr int kRowsMax = 14;    // rows per sub-tile (each lane keeps one field per row)
constexpr int kYStride = (kRowsMax + 3) & ~3;  // floats per trap in the staged row table (16-byte rows)
static_assert(kTileW == 32 && kYStride == 16, "16-byte staging of 32 columns and 16 rows per trap");
constexpr int kChunk = 128;     // traps whose tables are staged in shared memory at once
constexpr float kTwoPi = 6.283185307179586f;
constexpr int kModeAccurate = 0, kModeFast = 1, kModeSeparable = 2;  // kernel variants

// Work decomposition: the image is cut into 32-pixel-wide column strips; each strip's rows
// are dealt out as contiguous runs to a fixed number of resident blocks (one wave), so that
// every block gets the same number of row segments within one.  A block walks its run as
// sub-tiles of at most kRowsMax rows.
struct SubTile {
  int x0, y0, rows, pad;
};

struct StepArgs {
  int W, H, M;
  int chunk;              // traps staged in shared memory at once (1..kChunk)
  int copies;             // copies of each fixed-point accumulator buffer (a power of two; more than
                          // one in the separable mode only): block b adds into copy b % copies,
                          // spreading the atomics over more addresses
  int ldy4;               // row stride of Y4 (below)
  const SubTile *sub;     // work schedule: sub-tiles
  const int *first;       // [gridDim.x + 1]: block b processes sub-tiles first[b] .. first[b+1]-1
  const float *X;         // [M][W] column phase parts (turns if accurate, radians if fast)
  const float *Y;         // [M][H] row phase parts (same unit)
  const float *Y4;        // NULL, or [4][M][ldy4]: copy s holds Y shifted by s rows (Y4[s][m][i + s] =
                          // Y[m][i], zero elsewhere), so that every sub-tile's rows start 16-byte aligned
                          // in one of the copies
  const float2 *Xc;       // [M][W] e^{i 2pi X} (separable variant)
  const float2 *Yc;       // [2][M][ldy4] e^{i 2pi Y} (separable variant), in two copies: copy s holds the
                          // rows shifted by s (Yc[s][m][i + s] = e^{i 2pi Y_m(i)}, zero elsewhere), so
                          // that every sub-tile's rows start 16-byte aligned in one of them
  float *phi;             // [H*W] pixel phases, radians
  // BACK: weight update and coefficients from the previous launch's forward field
  const unsigned long long *acc_in;  // [copies][2][M] fixed-point sums of the previous forward: Re, Im
  const float *w_in;                 // [M] weights before this iteration's update
  float *w_out;                      // [M] updated weights (trap m written by block m % gridDim.x)
  // FWD: forward field of this launch's phases
  unsigned long long *acc_out;       // [copies][2][M] zero on entry (cleared by the launch before last)
  unsigned long long *acc_clear;     // [copies][2][M] cleared here for the next launch
  // Explicit coefficients G_m (Re, Im) instead of the GSW update (superposition, adjoint),
  // and the gradient output of the adjoint (ADJ)
  const float2 *G;                   // [M] or NULL: coefficients of the back-projection
  union {
    float *grad;  // [H*W] out: dL/dphi_j (ADJ)
    float2 *u;    // NULL, or [H*W]: unit phasors u_j of phi (gsw_once_kernel, see once_flags)
  };
  float inv_n;                       // 1 / N
  // gsw_once_kernel: its step takes u_j = S_j/|S_j| for the forward field and writes phi_j = arg S_j
  // only in the last launch of a call (kOnceLast), with u_j into u when set; its forward field of
  // the phases in phi reads u_j from u under kOnceReadU (the phasors the last step wrote for them)
  // instead of evaluating e^{i phi_j}.
  int once_flags;
  float *trace;                      // NULL, or out: e, u (Eq. 4) of the field this launch reads
  float fx_scale;           // 2^fx_shift: fixed-point scale of the sums
  float inv_fx_n;           // 1 / (N 2^fx_shift)
  float angle_units;        // 1 (radians) or 1/(2 pi) (turns): units of the tables
  float angle_eta;          // kFastEta (fast mode) or 0: relative scale added to angles in table units
};

__device__ __forceinline__ float sin_approx(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_approx(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The fast mode's angles are scaled by 1 + kFastEta before they reach sin.approx/cos.approx.
// Those instructions turn radians into revolutions with a multiplication by a rounded 1/(2 pi)
// that is rounded toward zero: on average the argument shrinks by 4.03e-8 (the constant) plus
// 2^-24 ln 2 = 4.13e-8 (the rounding, mean over a binade) of itself.  The scale is folded into
// the tables (FP64, when they are built), the pixel phases (once per pixel) and the
// coefficients' phases (once per trap), so it costs nothing per pair.  (What remains of the
// systematic part of the SFU's error is kept from adding up in the forward field by the
// per-sub-tile rotation of forward_traps.)
constexpr float kFastEta = 8.17e-8f;

// cos and sin of an angle given in table units: radians (fast, pre-scaled by 1 + kFastEta,
// |x| <= 3 pi here) or turns (accurate).
template <bool FAST>
__device__ __forceinline__ void cis(float x, float &co, float &si) {
  if (FAST) {
    si = sin_approx(x);
    co = cos_approx(x);
  } else {
    sincospif(2.0f * x, &si, &co);  // |x| <= 3/2 turns
  }
}

// A pixel phase (radians) in turns (the accurate mode's table units).
__device__ __forceinline__ float phase_turns(float ph) { return ph * 0.15915494309189535f; }

// A caller's pixel phase (any real value, radians) reduced to one turn, in turns.
__device__ __forceinline__ float reduced_phase_turns(float ph) {
  const float t = ph * 0.15915494309189535f;
  return t - rintf(t);
}

// A phase (radians) reduced to [-pi, pi] (two-part 2 pi).
__device__ __forceinline__ float reduced_radians(float ph) {
  const float k = rintf(ph * 0.15915494309189535f);
  return fmaf(-k, -1.74845553e-07f, fmaf(-k, 6.28318548e+00f, ph));
}

// The rotation theta in [-pi, pi) of a sub-tile of the fast forward field (see forward_traps),
// a fixed function of its position: a Weyl sequence (golden-ratio multiple, modulo 2^32) of the
// sub-tile's first pixel, so that neighbouring sub-tiles take well-spread angles.
__device__ __forceinline__ float subtile_rotation(const SubTile &st) {
  const unsigned h = ((unsigned)st.x0 * 65599u + (unsigned)st.y0) * 2654435769u;
  return (float)(h >> 8) * 3.7450018e-07f - 3.14159265f;  // 2 pi / 2^24
}

// e^{-i theta}, which undoes the rotation on the sub-tile's sums.
__device__ __forceinline__ float2 rotation_undo(float theta) {
  float s, c;
  sincosf(theta, &s, &c);
  return make_float2(c, -s);
}

// Fast mode: the forward field's pixel phase phi_j + theta (|phi_j| <= pi) in table units:
// reduced to [-pi, pi], scaled by 1 + kFastEta.
__device__ __forceinline__ float rotated_phase(float ph, float theta) {
  const float r = reduced_radians(ph + theta);
  return fmaf(r, kFastEta, r);
}


// Shared memory of a block: the staged tables of one trap chunk (X for the sub-tile's 32
// columns, Y for its rows, and the chunk's coefficients), the per-warp partial superpositions
// of half a sub-tile's rows, and the pixel phases of the sub-tile for the forward field.
constexpr int kHalfRows = kRowsMax / 2;
constexpr int kXsFloats = kChunk * kTileW;
constexpr int kYsFloats = kChunk * kYStride;
constexpr int kSmemBytes = (kXsFloats + kYsFloats) * 4 + kChunk * 8 + kWarps * kHalfRows * kTileW * 8 +
                           kRowsMax * kTileW * 4 + kChunk * 8;

__host__ __device__ constexpr int step_smem_bytes(int, bool) { return kSmemBytes; }

__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 4 : 0;  // 0 source bytes: the destination is zero-filled
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
// 16 bytes, both addresses 16-byte aligned (through L2 only).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialization
// may start while the previous kernel of the stream is still running; grid_dependency_wait()
// blocks until that kernel has finished and its writes are visible (a no-op otherwise), and
// allow_dependents() lets the next kernel start its own prologue early.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Groups: a block of the step kernel may hold several groups of kThreads threads, each acting
// as one block of the work schedule, a "virtual block" (see gsw_step_kernel).  With one group
// per block, gthread, vblock and vgrid are threadIdx.x, blockIdx.x and gridDim.x, and
// group_sync is a barrier of the whole block.
constexpr int kMaxGroups = 4;
__device__ __forceinline__ int gthread() { return threadIdx.x & (kThreads - 1); }
__device__ __forceinline__ int group_id() { return threadIdx.x / kThreads; }
__device__ __forceinline__ int vblock() { return blockIdx.x * (blockDim.x / kThreads) + group_id(); }
__device__ __forceinline__ int vgrid() { return gridDim.x * (blockDim.x / kThreads); }
__device__ __forceinline__ void group_sync() {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + group_id()), "n"(kThreads) : "memory");
}

// Traps [lo, hi) of a staged chunk of n that warp `warp` of a group takes.  Warps w and w + 4
// issue to the same SM sub-partition (warp slot mod 4) and share its special-function unit, so
// each such pair takes one quarter of the chunk, split between its two warps: every
// sub-partition gets the same number of traps to within one (with M = 100 a plain eighth split
// gives two sub-partitions 26 traps and two 24).
__device__ __forceinline__ void warp_traps(int n, int warp, int &lo, int &hi) {
  const int s = warp & 3, q0 = s * n / 4, q1 = (s + 1) * n / 4, mid = (q0 + q1) >> 1;
  lo = warp < 4 ? q0 : mid;
  hi = warp < 4 ? mid : q1;
}

// The field V_m of the previous forward, from its fixed-point sums; MULTI: added over the
// copies (integer addition, exact in any order).  The direct kernels run with one copy.
template <bool MULTI = false>
__device__ __forceinline__ float2 field_from_sums(const StepArgs &a, int m) {
  long long sr = (long long)__ldcg(a.acc_in + m), si = (long long)__ldcg(a.acc_in + a.M + m);
  if (MULTI)
#pragma unroll 7
    for (int c = 1; c < a.copies; c++) {
      sr += (long long)__ldcg(a.acc_in + (size_t)c * 2 * a.M + m);
      si += (long long)__ldcg(a.acc_in + (size_t)c * 2 * a.M + a.M + m);
    }
  return make_float2((float)sr * a.inv_fx_n, (float)si * a.inv_fx_n);
}

// The accumulator copy this block adds its forward sums into (copies is a power of two).
__device__ __forceinline__ unsigned long long *block_acc(const StepArgs &a) {
  return a.acc_out + (size_t)((unsigned)vblock() & (unsigned)(a.copies - 1)) * 2 * a.M;
}

// |v|^2 with its rounding fixed in the source (v.y^2 rounded, then one fused multiply-add), so
// that every kernel that inlines it computes the same bits whatever the compiler would fuse.
__device__ __forceinline__ float abs2(float2 v) { return fmaf(v.x, v.x, v.y * v.y); }

// Sec. 3 weight update and back-projection coefficient of a trap with field v and weight w:
// w <- w <|V|>/|V_m|; if |V_m| < 1e-30 the unit field is 1 and w stays.  Polar form
// (w', arg V_m in table units: times units, plus eta of itself), or complex form w' V_m/|V_m|
// (COMPLEX).
template <bool COMPLEX>
__device__ __forceinline__ float2 update_from(float2 v, float w, float mean, float units, float eta = 0.f) {
  const float am = sqrtf(abs2(v));
  if (COMPLEX) {
    if (am < 1e-30f) return make_float2(w, 0.f);
    const float s = w * mean / (am * am);
    return make_float2(s * v.x, s * v.y);
  }
  if (am >= 1e-30f) w = w * mean / am;
  const float ang = atan2f(v.y, v.x);
  return make_float2(w, am >= 1e-30f ? fmaf(ang, eta, ang * units) : 0.f);
}

// The coefficient of trap m from the previous forward's sums and weights (both written by
// other blocks: read from L2, not from a possibly stale L1 line).
__device__ __forceinline__ float2 coefficient(const StepArgs &a, int m, float mean) {
  return update_from<false>(field_from_sums(a, m), __ldcg(a.w_in + m), mean, a.angle_units, a.angle_eta);
}

// Explicit coefficient of trap m (superposition or adjoint) in polar form (|G_m|, arg G_m).
__device__ __forceinline__ float2 adjoint_coefficient(const StepArgs &a, int m) {
  const float2 g = a.G[m];
  const float ang = atan2f(g.y, g.x);
  return make_float2(sqrtf(abs2(g)), fmaf(ang, a.angle_eta, ang * a.angle_units));
}

// Stages, with asynchronous copies (all in flight at once), the X (32 columns from x0) and Y
// (rows y0 .. y0+rows-1) tables of traps [m0, m0+n), plus their coefficients when BACK
// (GSW coefficients, or adjoint coefficients when ADJ).
// The caller synchronises the block afterwards.
// A trap's 32 columns of the X table are copied as 8 16-byte pieces when W is a multiple of 4
// (rows then start 16-byte aligned; x0 is a multiple of 32) and the strip lies inside the image;
// otherwise column by column, zero past the right edge.  (Four times fewer copy instructions: the
// staging of every chunk is on the sub-tile's critical path.)
template <bool BACK, bool ADJ = false>
__device__ __forceinline__ void stage_tables(const StepArgs &a, int m0, int n, const SubTile &st,
                                             float *Xs, float *Ys, float2 *Cs, bool xy = true,
                                             float mean = 0.f, bool coef = true) {
  if (xy && (a.W & 3) == 0 && st.x0 + kTileW <= a.W) {
    for (int i = gthread(); i < n * (kTileW / 4); i += kThreads) {
      const int k = i >> 3, q = i & 7;
      cp_async16(Xs + k * kTileW + 4 * q, a.X + (size_t)(m0 + k) * a.W + st.x0 + 4 * q);
    }
  } else {
    for (int i = gthread(); xy && i < n * kTileW; i += kThreads) {
      const int k = i / kTileW, col = st.x0 + (i % kTileW);
      const bool ok = col < a.W;
      cp_async4(Xs + i, a.X + (ok ? (size_t)(m0 + k) * a.W + col : 0), ok);
    }
  }
  if (xy && a.Y4) {  // the trap's kYStride rows from y0 as 4 16-byte pieces of the aligned copy
    const int s = (4 - (st.y0 & 3)) & 3;
    const float *src = a.Y4 + ((size_t)s * a.M + m0) * a.ldy4 + st.y0 + s;
    for (int i = gthread(); i < n * (kYStride / 4); i += kThreads) {
      const int k = i >> 2, q = i & 3;
      cp_async16(Ys + k * kYStride + 4 * q, src + (size_t)k * a.ldy4 + 4 * q);
    }
  } else {
    for (int i = gthread(); xy && i < n * kYStride; i += kThreads) {
      const int k = i / kYStride, r = i % kYStride;
      const bool ok = r < st.rows;
      cp_async4(Ys + i, a.Y + (ok ? (size_t)(m0 + k) * a.H + st.y0 + r : 0), ok);
    }
  }
  if (BACK && coef)
    for (int i = gthread(); i < n; i += kThreads)
      Cs[i] = (ADJ || a.G) ? adjoint_coefficient(a, m0 + i) : coefficient(a, m0 + i, mean);
  cp_async_wait_all();
}

constexpr int kGroup = 8;  // traps reduced together over the lanes of a warp
// ... in the direct kernels' forward field (4 or 8: the unrolled loop body over a group's traps
// and the sub-tile's rows is the largest code of the kernel)
constexpr int kFwdGroup = 8;

// Sums acc[0..7] over the 32 lanes of a warp with 18 shuffles instead of 8 x 5: at each of
// the first three steps a lane keeps half of its traps and sends the other half to its
// partner, so that after offsets 16, 8, 4 lane l holds trap (l >> 2) & 7 summed over 8 lanes;
// two butterfly steps finish the sum.  Returns the total of trap (lane >> 2) & 7 (exact
// same value in every run; lanes with (lane & 3) == 0 are the ones that store it).
__device__ __forceinline__ float2 warp_reduce8(float2 (&acc)[kGroup], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const float2 send = b4 ? acc[i] : acc[i + 4], keep = b4 ? acc[i + 4] : acc[i];
    acc[i].x = keep.x + __shfl_xor_sync(0xffffffffu, send.x, 16);
    acc[i].y = keep.y + __shfl_xor_sync(0xffffffffu, send.y, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; i++) {
    const float2 send = b3 ? acc[i] : acc[i + 2], keep = b3 ? acc[i + 2] : acc[i];
    acc[i].x = keep.x + __shfl_xor_sync(0xffffffffu, send.x, 8);
    acc[i].y = keep.y + __shfl_xor_sync(0xffffffffu, send.y, 8);
  }
  {
    const float2 send = b2 ? acc[0] : acc[1], keep = b2 ? acc[1] : acc[0];
    acc[0].x = keep.x + __shfl_xor_sync(0xffffffffu, send.x, 4);
    acc[0].y = keep.y + __shfl_xor_sync(0xffffffffu, send.y, 4);
  }
  float2 v = acc[0];
  v.x += __shfl_xor_sync(0xffffffffu, v.x, 2);
  v.y += __shfl_xor_sync(0xffffffffu, v.y, 2);
  v.x += __shfl_xor_sync(0xffffffffu, v.x, 1);
  v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
  return v;
}

// Sums acc[0..3] over the 32 lanes of a warp with 12 shuffles: at offsets 16 and 8 a lane keeps
// half of its traps and sends the other half, so that lane l then holds trap (l >> 3) & 3 summed
// over 4 lanes; three butterfly steps finish the sum (lanes with (lane & 7) == 0 store it).
__device__ __forceinline__ float2 warp_reduce4(float2 (&acc)[4], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8;
#pragma unroll
  for (int i = 0; i < 2; i++) {
    const float2 send = b4 ? acc[i] : acc[i + 2], keep = b4 ? acc[i + 2] : acc[i];
    acc[i].x = keep.x + __shfl_xor_sync(0xffffffffu, send.x, 16);
    acc[i].y = keep.y + __shfl_xor_sync(0xffffffffu, send.y, 16);
  }
  {
    const float2 send = b3 ? acc[0] : acc[1], keep = b3 ? acc[1] : acc[0];
    acc[0].x = keep.x + __shfl_xor_sync(0xffffffffu, send.x, 8);
    acc[0].y = keep.y + __shfl_xor_sync(0xffffffffu, send.y, 8);
  }
  float2 v = acc[0];
#pragma unroll
  for (int o = 4; o; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// The group reductions by size, and the trap of the group whose total lane `lane` holds.
__device__ __forceinline__ float2 warp_reduce_group(float2 (&acc)[8], int lane) { return warp_reduce8(acc, lane); }
__device__ __forceinline__ float2 warp_reduce_group(float2 (&acc)[4], int lane) { return warp_reduce4(acc, lane); }
template <int NG>
__device__ __forceinline__ int group_trap(int lane) { return (lane >> (NG == 8 ? 2 : 3)) & (NG - 1); }

// Back-projection of traps [lo, hi) of the staged chunk onto the R rows of this lane:
// S_r += w_m e^{i (X_m + Y_m(r) + arg V_m)}.  R is a compile-time row count.
template <bool FAST, int R>
__device__ __forceinline__ void back_traps(const float *Xs, const float *Ys, const float2 *Cs, int lo, int hi,
                                           int lane, float2 (&S)[kRowsMax]) {
  for (int k = lo; k < hi; k++) {
    const float2 c = Cs[k];                      // (w_m, arg V_m)
    const float xm = Xs[k * kTileW + lane] + c.y;
    const float4 *yq = reinterpret_cast<const float4 *>(Ys + k * kYStride);
#pragma unroll
    for (int q = 0; q < (R + 3) / 4; q++) {
      const float4 y4 = yq[q];
      const float yy[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int r = 4 * q + j;
        if (r < R) {
          float co, si;
          cis<FAST>(xm + yy[j], co, si);
          S[r].x = fmaf(c.x, co, S[r].x);
          S[r].y = fmaf(c.x, si, S[r].y);
        }
      }
    }
  }
}

// Forward field (Eq. 1) of traps [lo, hi) of the staged chunk over the R rows of this lane's
// column: sum_r e^{i (phi_r - X_m - Y_m(r))}, summed over the warp 8 traps at a time and
// added, in fixed point, to acc_out[m0 + k] (Re) and acc_out[M + m0 + k] (Im).  ph holds the lane's
// pixel phases in table units; msk is 1 for a lane inside the image, 0 past its right edge.
// Fast mode: ph holds phi_r + theta, theta a rotation fixed per sub-tile, and each trap's sum
// over the sub-tile is multiplied by undo = e^{-i theta} before it is added (4 FP32 operations
// per trap and sub-tile).  The SFU's error has a systematic part: measured on GB300, fields of
// random phases evaluated without the rotation carry an offset of ~1e-8 on every trap, the same
// for all traps (their arguments phi_j - Delta_j^m are spread alike), ~1e-4 of the weakest
// |V_m| on a 512^2 SLM.  With the rotation, the offset of each sub-tile's sum turns by its own
// angle -theta, and over the sub-tiles those contributions cancel instead of adding up.
template <bool FAST, int R>
__device__ __forceinline__ void forward_traps(const float *Xs, const float *Ys, int lo, int hi, int lane,
                                              const float (&ph)[kRowsMax], float msk, const StepArgs &a,
                                              int m0, float2 undo = make_float2(1.f, 0.f)) {
  constexpr int NG = kFwdGroup;
  static_assert(NG == 4 || NG == 8, "forward group of 4 or 8 traps");
  for (int g = lo; g < hi; g += NG) {
    float2 acc[NG];
#pragma unroll
    for (int i = 0; i < NG; i++) {
      acc[i] = make_float2(0.f, 0.f);
      const int k = g + i;
      if (k < hi) {
        const float xm = Xs[k * kTileW + lane];
        const float4 *yq = reinterpret_cast<const float4 *>(Ys + k * kYStride);
#pragma unroll
        for (int q = 0; q < (R + 3) / 4; q++) {
          const float4 y4 = yq[q];
          const float yy[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
          for (int j = 0; j < 4; j++) {
            const int r = 4 * q + j;
            if (r < R) {
              float co, si;
              cis<FAST>((ph[r] - yy[j]) - xm, co, si);
              acc[i].x = fmaf(msk, co, acc[i].x);
              acc[i].y = fmaf(msk, si, acc[i].y);
            }
          }
        }
      }
    }
    float2 v = warp_reduce_group(acc, lane);
    const int k = g + group_trap<NG>(lane);
    const bool store = (lane & (32 / NG - 1)) == 0;
    if (FAST) v = make_float2(fmaf(v.x, undo.x, -v.y * undo.y), fmaf(v.x, undo.y, v.y * undo.x));
    if (store && k < hi) {
      // |v| <= 32 * kRowsMax, so v * 2^fx_shift is an exact integer far below 2^63
      atomicAdd(a.acc_out + m0 + k, (unsigned long long)__float2ll_rn(v.x * a.fx_scale));
      atomicAdd(a.acc_out + a.M + m0 + k, (unsigned long long)__float2ll_rn(v.y * a.fx_scale));
    }
  }
}

// Float-float ("double-single") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2.
// TwoSum (Knuth) and FastTwoSum (Dekker) give the exact rounding error of one addition.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b.hi - bb);
  const float e = err + (a.lo + b.lo);
  const float hi = s + e;
  return {hi, e - (hi - s)};
}

// Weight update a thread writes after its block's work (prefetched in the prologue).
struct LateWeight {
  int own;   // the block's first trap (own + stride * t for thread t); >= M: the block owns none
  int m;     // this thread's first trap (m >= M: none)
  float2 v;  // its field
  float w;   // its weight before the update
  ff part;   // this thread's share of sum_m |V_m| (traps t, t + kThreads, ...)
};

// Start of a GSW step: the previous forward's fields are read once, every load issued before
// any is used.  Writes the coefficients of traps [0, mc) into C0 (polar, or complex when
// COMPLEX) without the factor <|V|> of the weight update: a factor common to all coefficients
// scales S_j and leaves arg S_j unchanged (the weights' global scale is free, reading R6), so
// no block-wide reduction stands between the sums and the back-projection.  Keeps in lw the
// thread's share of sum |V_m| and the prefetched weight of trap own + stride * gthread(),
// which write_weights completes after the block's work.
// trace: NULL, or where block 0 writes e and u (Eq. 4) of the fields it read (convergence trace).
template <bool COMPLEX>
__device__ __forceinline__ void gsw_prologue(const StepArgs &a, int mc, float2 *C0, int own, int stride,
                                             LateWeight &lw, float *trace = nullptr) {
  const int t = gthread();
  lw.own = own;
  lw.m = own + stride * t;
  lw.v = make_float2(0.f, 0.f);
  lw.w = 0.f;
  if (lw.m < a.M) {
    lw.v = field_from_sums<COMPLEX>(a, lw.m);
    lw.w = __ldcg(a.w_in + lw.m);
  }
  const float w0 = t < mc ? __ldcg(a.w_in + t) : 0.f;
  float2 v0 = make_float2(0.f, 0.f);
  ff s = {0.f, 0.f};
  const bool tr = trace && vblock() == 0;
  ff si = {0.f, 0.f};
  float mx = -1.f, mn = 3.0e38f;
  for (int m = t; m < a.M; m += kThreads) {
    const float2 v = field_from_sums<COMPLEX>(a, m);
    if (m == t) v0 = v;
    s = ff_add(s, {sqrtf(abs2(v)), 0.f});
    if (tr) {
      const float I = abs2(v);
      si = ff_add(si, {I, 0.f});
      mx = fmaxf(mx, I);
      mn = fminf(mn, I);
    }
  }
  lw.part = s;
  if (t < mc) C0[t] = update_from<COMPLEX>(v0, w0, 1.f, a.angle_units, a.angle_eta);
  if (tr) {  // virtual block 0 only: e = sum I_m, u = 1 - (max - min)/(max + min) of the fields read
    __shared__ ff tpart[kWarps];
    __shared__ float ext[2][kWarps];  // (group 0 of block 0 alone uses these)
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      si = ff_add(si, {__shfl_down_sync(0xffffffffu, si.hi, o), __shfl_down_sync(0xffffffffu, si.lo, o)});
      mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
      mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
    }
    if ((t & 31) == 0) {
      tpart[t >> 5] = si;
      ext[0][t >> 5] = mx;
      ext[1][t >> 5] = mn;
    }
    group_sync();
    if (t == 0) {
      ff e = tpart[0];
      float hi = ext[0][0], lo = ext[1][0];
      for (int i = 1; i < kWarps; i++) {
        e = ff_add(e, tpart[i]);
        hi = fmaxf(hi, ext[0][i]);
        lo = fminf(lo, ext[1][i]);
      }
      trace[0] = e.hi + e.lo;
      trace[1] = (hi + lo > 0.f) ? 1.f - (hi - lo) / (hi + lo) : 0.f;
    }
  }
}

// After the block's work, in blocks that own weights (a block-uniform condition): <|V|> (mean
// of |V_m| over the traps, Sec. 3) from the threads' shares in one fixed order (warp
// shuffles, warps in order), so every such block obtains the same bits, and the block's
// weight updates w_m <- w_m <|V|>/|V_m| (traps lw.m, lw.m + stride * kThreads, ...).
template <bool MULTI = false>
__device__ __forceinline__ void write_weights(const StepArgs &a, const LateWeight &lw, int stride) {
  if (lw.own >= a.M) return;
  __shared__ ff parts[kMaxGroups][kWarps];
  ff *const part = parts[group_id()];
  ff s = lw.part;
#pragma unroll
  for (int o = 16; o; o >>= 1)
    s = ff_add(s, {__shfl_down_sync(0xffffffffu, s.hi, o), __shfl_down_sync(0xffffffffu, s.lo, o)});
  group_sync();
  if ((gthread() & 31) == 0) part[gthread() >> 5] = s;
  group_sync();
  ff q = part[0];
#pragma unroll
  for (int i = 1; i < kWarps; i++) q = ff_add(q, part[i]);
  const float mean = (q.hi + q.lo) / (float)a.M;
  if (lw.m < a.M) a.w_out[lw.m] = update_from<false>(lw.v, lw.w, mean, 1.f).x;
  for (int m = lw.m + stride * kThreads; m < a.M; m += stride * kThreads)
    a.w_out[m] = update_from<false>(field_from_sums<MULTI>(a, m), __ldcg(a.w_in + m), mean, 1.f).x;
}

struct FinalizeArgs {
  int M;
  int copies;                     // accumulator copies (as StepArgs::copies)
  const unsigned long long *acc;  // [copies][2][M] sums of the last forward field
  unsigned long long *acc_all;    // [3][copies][2][M] all accumulators: cleared for the next call
  const float *w_src;             // [M] weights after the last update
  float *w_dst;                   // [M] where the weights live between calls (may equal w_src)
  long long *Vsum;                // [2][M] out: the sums (V_m = Vsum / (N 2^fx_shift))
  float *metrics;                 // [2] out: e, u (Eq. 4)
  float inv_fx_n;
  unsigned long long *done;       // NULL, or out: %globaltimer (ns) when the hologram completed
};

constexpr int kFinalizeThreads = 1024;

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One block, once per hot_gsw call: efficiency e = sum |V_m|^2 and uniformity
// u = 1 - (max I - min I)/(max I + min I) (Eq. 4) of the final forward field (fixed order),
// the field sums for the caller, the weights back into their home buffer, and every
// accumulator cleared.
__device__ __forceinline__ void finalize_block(const FinalizeArgs &a) {
  struct Part {
    ff si;
    float mx, mn;
  };
  __shared__ Part part[kFinalizeThreads / 32];
  Part p = {{0.f, 0.f}, -1.f, 3.0e38f};
  for (int m = threadIdx.x; m < a.M; m += kFinalizeThreads) {
    long long sr = 0, si = 0;
    for (int c = 0; c < a.copies; c++) {
      sr += (long long)__ldcg(a.acc + (size_t)c * 2 * a.M + m);
      si += (long long)__ldcg(a.acc + (size_t)c * 2 * a.M + a.M + m);
    }
    a.Vsum[m] = sr;
    a.Vsum[a.M + m] = si;
    const float vr = (float)sr * a.inv_fx_n, vi = (float)si * a.inv_fx_n;
    const float I = vr * vr + vi * vi;
    p.si = ff_add(p.si, {I, 0.f});
    p.mx = fmaxf(p.mx, I);
    p.mn = fminf(p.mn, I);
    if (a.w_dst != a.w_src) a.w_dst[m] = a.w_src[m];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    p.si = ff_add(p.si, {__shfl_down_sync(0xffffffffu, p.si.hi, o), __shfl_down_sync(0xffffffffu, p.si.lo, o)});
    p.mx = fmaxf(p.mx, __shfl_down_sync(0xffffffffu, p.mx, o));
    p.mn = fminf(p.mn, __shfl_down_sync(0xffffffffu, p.mn, o));
  }
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = p;
  __syncthreads();  // every read of the accumulators is done before they are cleared
  for (int i = threadIdx.x; i < 6 * a.M * a.copies; i += kFinalizeThreads) a.acc_all[i] = 0ull;
  if (threadIdx.x == 0) {
    Part q = part[0];
    for (int i = 1; i < kFinalizeThreads / 32; i++) {
      q.si = ff_add(q.si, part[i].si);
      q.mx = fmaxf(q.mx, part[i].mx);
      q.mn = fminf(q.mn, part[i].mn);
    }
    a.metrics[0] = q.si.hi + q.si.lo;
    a.metrics[1] = (q.mx + q.mn > 0.f) ? 1.f - (q.mx - q.mn) / (q.mx + q.mn) : 0.f;
  }
}

static __global__ void __launch_bounds__(kFinalizeThreads) gsw_finalize_kernel(FinalizeArgs a) {
  grid_dependency_wait();
  finalize_block(a);
}

// Batched: block h finalizes hologram h and stamps its completion time.
static __global__ void __launch_bounds__(kFinalizeThreads) gsw_finalize_batch_kernel(const FinalizeArgs *args) {
  grid_dependency_wait();
  const FinalizeArgs &a = args[blockIdx.x];
  finalize_block(a);
  __syncthreads();
  if (threadIdx.x == 0 && a.done) {
    __threadfence();
    *a.done = global_timer_ns();
  }
}

// Calls BODY with the compile-time constant R equal to the runtime value rows (1..kRowsMax).
#define HOT_WITH_ROWS(rows, BODY)              \
  switch (rows) {                              \
    case 1: { constexpr int R = 1; BODY; } break;   \
    case 2: { constexpr int R = 2; BODY; } break;   \
    case 3: { constexpr int R = 3; BODY; } break;   \
    case 4: { constexpr int R = 4; BODY; } break;   \
    case 5: { constexpr int R = 5; BODY; } break;   \
    case 6: { constexpr int R = 6; BODY; } break;   \
    case 7: { constexpr int R = 7; BODY; } break;   \
    case 8: { constexpr int R = 8; BODY; } break;   \
    case 9: { constexpr int R = 9; BODY; } break;   \
    case 10: { constexpr int R = 10; BODY; } break; \
    case 11: { constexpr int R = 11; BODY; } break; \
    case 12: { constexpr int R = 12; BODY; } break; \
    case 13: { constexpr int R = 13; BODY; } break; \
    default: { constexpr int R = 14; BODY; } break; \
  }
static_assert(kRowsMax == 14, "HOT_WITH_ROWS covers 1..14 rows");
static_assert(kRowsMax % 2 == 0 && kRowsMax / 2 <= kWarps, "each warp finishes one row per half of a sub-tile");

// Persistent blocks, one wave; the 8 warps of a block split the traps of each chunk.
// BACK: weight update and back-projection -> a.phi.  FWD: forward field of the sub-tile phases.
// ADJ (with BACK, without FWD): the adjoint of Eq. 1 instead -- the same superposition with
// coefficients G_m, S_j = sum_m G_m e^{i Delta_j^m}, written as the gradient
// dL/dphi_j = (1/N) Im[e^{-i phi_j} S_j] of a real loss L(V) (a.phi is read, not written).
// Shared-memory views of a step block.
struct StepSmem {
  float *Xs, *Ys;
  float2 *Cs, *Sp;
  float *Ps;
  float2 *C0;  // [kChunk] coefficients of the first trap chunk, from the step's prologue
  __device__ __forceinline__ explicit StepSmem(unsigned char *raw) {
    Xs = reinterpret_cast<float *>(raw);
    Ys = Xs + kXsFloats;
    Cs = reinterpret_cast<float2 *>(Ys + kYsFloats);
    Sp = Cs + kChunk;                                                  // [kWarps][kHalfRows][kTileW]
    Ps = reinterpret_cast<float *>(Sp + kWarps * kHalfRows * kTileW);  // [kRowsMax][kTileW] phases
    C0 = reinterpret_cast<float2 *>(Ps + kRowsMax * kTileW);
  }
};

// One sub-tile of the hologram a: back-projection (with the coefficients implied by `mean`,
// or explicit ones) and/or forward field.  prestaged: the first chunk's X/Y tables are
// already in shared memory (staged in the prologue) -- cleared after use.  C0: the first
// chunk's coefficients, computed by the step's prologue (NULL: staged with the tables).
template <bool FAST, bool BACK, bool FWD, bool ADJ>
__device__ __forceinline__ void process_subtile(const StepArgs &a, const SubTile st, float mean, bool &prestaged,
                                                const StepSmem &sm, const float2 *C0 = nullptr) {
  const int lane = threadIdx.x & 31, warp = gthread() >> 5;
  const int mc = a.M < a.chunk ? a.M : a.chunk;
  const int nchunks = (a.M + mc - 1) / mc;
  const int ix = st.x0 + lane;
  const bool col_ok = ix < a.W;

  if (BACK) {
    float2 S[kRowsMax];
#pragma unroll
    for (int r = 0; r < kRowsMax; r++) S[r] = make_float2(0.f, 0.f);
    for (int ch = 0; ch < nchunks; ch++) {
      const int m0 = ch * mc, n = min(mc, a.M - m0);
      const bool pre = C0 && ch == 0;
      group_sync();  // earlier readers of the tables are done
      stage_tables<true, ADJ>(a, m0, n, st, sm.Xs, sm.Ys, sm.Cs, !prestaged, mean, !pre);
      prestaged = false;
      group_sync();
      int lo, hi;
      warp_traps(n, warp, lo, hi);
      const float2 *C = pre ? C0 : sm.Cs;
      HOT_WITH_ROWS(st.rows, (back_traps<FAST, R>(sm.Xs, sm.Ys, C, lo, hi, lane, S)));
    }
    // Sum the 8 warps' superpositions, half of the rows at a time, in warp order.
#pragma unroll
    for (int h = 0; h < 2; h++) {
      if (h * kHalfRows >= st.rows) break;
      group_sync();  // Sp and the phase rows are free
#pragma unroll
      for (int i = 0; i < kHalfRows; i++)
        if (h * kHalfRows + i < st.rows) sm.Sp[(warp * kHalfRows + i) * kTileW + lane] = S[h * kHalfRows + i];
      group_sync();
      if (warp < kHalfRows && h * kHalfRows + warp < st.rows) {
        const int r = h * kHalfRows + warp;
        float2 s = sm.Sp[warp * kTileW + lane];
#pragma unroll
        for (int w = 1; w < kWarps; w++) {
          const float2 q = sm.Sp[(w * kHalfRows + warp) * kTileW + lane];
          s.x += q.x;
          s.y += q.y;
        }
        const size_t j = (size_t)(st.y0 + r) * a.W + ix;
        if (ADJ) {
          if (col_ok) {
            float sp, cp;
            sincosf(a.phi[j], &sp, &cp);
            a.grad[j] = (cp * s.y - sp * s.x) * a.inv_n;  // Im[(cos - i sin)(S.x + i S.y)] / N
          }
        } else {
          const float ph = atan2f(s.y, s.x);
          if (col_ok) a.phi[j] = ph;
          if (FWD) sm.Ps[r * kTileW + lane] = FAST ? rotated_phase(ph, subtile_rotation(st)) : phase_turns(ph);
        }
      }
    }
  } else if (FWD) {
    group_sync();  // earlier readers of the phases and of the tables are done
    for (int r = warp; r < st.rows; r += kWarps) {
      const float ph = col_ok ? a.phi[(size_t)(st.y0 + r) * a.W + ix] : 0.0f;
      sm.Ps[r * kTileW + lane] = FAST ? rotated_phase(reduced_radians(ph), subtile_rotation(st)) : reduced_phase_turns(ph);
    }
  }

  if (FWD) {
    const float2 undo = FAST ? rotation_undo(subtile_rotation(st)) : make_float2(1.f, 0.f);
    group_sync();  // the phases are complete
    float ph[kRowsMax];
#pragma unroll
    for (int r = 0; r < kRowsMax; r++) ph[r] = r < st.rows ? sm.Ps[r * kTileW + lane] : 0.0f;
    for (int ch = 0; ch < nchunks; ch++) {
      const int m0 = ch * mc, n = min(mc, a.M - m0);
      if (!BACK || nchunks > 1) {  // with one chunk the back-projection's tables are still staged
        if (ch) group_sync();
        stage_tables<false>(a, m0, n, st, sm.Xs, sm.Ys, sm.Cs);
        group_sync();
      }
      int lo, hi;
      warp_traps(n, warp, lo, hi);
      HOT_WITH_ROWS(st.rows, (forward_traps<FAST, R>(sm.Xs, sm.Ys, lo, hi, lane, ph, col_ok ? 1.f : 0.f, a, m0, undo)));
    }
  }
}

// GROUPS > 1: blocks of GROUPS x kThreads threads (4 / GROUPS per SM), group g of block b acting
// as virtual block GROUPS b + g of the schedule, with its own shared memory and barrier.  The
// schedule deals consecutive runs of row segments to consecutive virtual blocks, and consecutive
// runs add up to their equal share to within one segment: with GROUPS = 4 an SM holds its equal
// share, with GROUPS = 2 each of its two blocks does, whereas with independent blocks an SM may
// hold four runs that are all one segment longer than average.
template <bool FAST, bool BACK, bool FWD, bool ADJ = false, int GROUPS = 1>
__global__ void __launch_bounds__(kThreads * GROUPS, kMaxGroups / GROUPS) gsw_step_kernel(StepArgs a) {
  static_assert(!ADJ || (BACK && !FWD), "the adjoint is a back-projection without forward field");
  static_assert(GROUPS >= 1 && GROUPS <= kMaxGroups, "groups per block");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const StepSmem sm(smem_raw + (GROUPS > 1 ? group_id() * kSmemBytes : 0));
  const int mc = a.M < a.chunk ? a.M : a.chunk;
  const int vb = vblock(), vg = vgrid();
  const int t_begin = a.first[vb], t_end = a.first[vb + 1];

  // Prologue, overlapping the previous kernel: the trap tables are constant during hot_gsw,
  // so the first chunk of the back-projection is staged before waiting for its field sums.
  allow_dependents();
  bool prestaged = false;
  if (BACK && t_begin < t_end) {
    const SubTile st0 = a.sub[t_begin];
    stage_tables<false>(a, 0, mc, st0, sm.Xs, sm.Ys, sm.Cs);
    prestaged = true;
  }
  grid_dependency_wait();
  if (FWD)  // the buffer the next launch accumulates into
    for (int i = vb * kThreads + gthread(); i < 2 * a.M * a.copies; i += vg * kThreads) a.acc_clear[i] = 0ull;
  LateWeight lw;
  const bool gsw = BACK && !ADJ && !a.G;
  if (gsw) gsw_prologue<false>(a, mc, sm.C0, vb, vg, lw, a.trace);
  for (int t = t_begin; t < t_end; t++)
    process_subtile<FAST, BACK, FWD, ADJ>(a, a.sub[t], 1.f, prestaged, sm, gsw ? sm.C0 : nullptr);
  if (gsw) write_weights(a, lw, vg);
}

// Start stamp of a batched sequence (%globaltimer, ns).
static __global__ void stamp_kernel(unsigned long long *t) { *t = global_timer_ns(); }

// The trap-intensity loss of the differentiable form and its adjoint coefficients, from the
// forward field's fixed-point sums: I_m = |V_m|^2 (the intensities of Eq. 4),
//   L = -sum_m log I_m + beta var_m(I)   (population variance),
//   G_m = 2 dL/d conj(V_m) = 2 g_m V_m,  g_m = dL/dI_m = -1/I_m + beta (2/M)(I_m - mean I),
// the coefficients of the adjoint superposition (hot_field_adjoint) that gives dL/dphi.  One
// block; FP64 sums in a fixed order (threads, then warps in order).  Like gsw_finalize_kernel it
// also leaves the sums for the caller, e and u, and clears the accumulators.
struct LossArgs {
  int M, copies;
  const unsigned long long *acc;  // [copies][2][M] sums of the forward field
  unsigned long long *acc_all;    // [3][copies][2][M]: cleared
  long long *Vsum;                // [2][M] out
  float *metrics;                 // [2] out: e, u
  double inv_fx_n;                // 1 / (N 2^fx_shift)
  double beta;
  float2 *G;                      // [M] out
  float *loss;                    // [1] out
};

constexpr int kLossThreads = 1024;

// Sum over the block in a fixed order; every thread gets the total.
__device__ __forceinline__ double block_sum(double v, double *part) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();  // earlier readers of part are done
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < kLossThreads / 32; i++) t += part[i];
  return t;
}

static __global__ void __launch_bounds__(kLossThreads) intensity_loss_kernel(LossArgs a) {
  __shared__ double part[kLossThreads / 32];
  __shared__ float ext[2][kLossThreads / 32];
  double sI = 0.0, sLog = 0.0;
  float mx = -1.f, mn = 3.0e38f;
  for (int m = threadIdx.x; m < a.M; m += kLossThreads) {
    long long sr = 0, si = 0;
    for (int c = 0; c < a.copies; c++) {
      sr += (long long)a.acc[(size_t)c * 2 * a.M + m];
      si += (long long)a.acc[(size_t)c * 2 * a.M + a.M + m];
    }
    a.Vsum[m] = sr;
    a.Vsum[a.M + m] = si;
    const double vr = (double)sr * a.inv_fx_n, vi = (double)si * a.inv_fx_n, I = vr * vr + vi * vi;
    sI += I;
    sLog += log(I);
    mx = fmaxf(mx, (float)I);
    mn = fminf(mn, (float)I);
  }
  const double e = block_sum(sI, part), slog = block_sum(sLog, part);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    ext[0][threadIdx.x >> 5] = mx;
    ext[1][threadIdx.x >> 5] = mn;
  }
  const double mean = e / a.M;
  double sVar = 0.0;
  for (int m = threadIdx.x; m < a.M; m += kLossThreads) {
    const double vr = (double)a.Vsum[m] * a.inv_fx_n, vi = (double)a.Vsum[a.M + m] * a.inv_fx_n;
    const double d = vr * vr + vi * vi - mean;
    sVar += d * d;
  }
  const double var = block_sum(sVar, part) / a.M;  // (its barriers also order ext and Vsum)
  for (int m = threadIdx.x; m < a.M; m += kLossThreads) {
    const double vr = (double)a.Vsum[m] * a.inv_fx_n, vi = (double)a.Vsum[a.M + m] * a.inv_fx_n;
    const double I = vr * vr + vi * vi;
    const double g = -1.0 / I + a.beta * (2.0 / a.M) * (I - mean);
    a.G[m] = make_float2((float)(2.0 * g * vr), (float)(2.0 * g * vi));
  }
  for (int i = threadIdx.x; i < 6 * a.M * a.copies; i += kLossThreads) a.acc_all[i] = 0ull;
  if (threadIdx.x == 0) {
    float hi = ext[0][0], lo = ext[1][0];
    for (int i = 1; i < kLossThreads / 32; i++) {
      hi = fmaxf(hi, ext[0][i]);
      lo = fminf(lo, ext[1][i]);
    }
    *a.loss = (float)(-slog + a.beta * var);
    a.metrics[0] = (float)e;
    a.metrics[1] = (hi + lo > 0.f) ? 1.f - (hi - lo) / (hi + lo) : 0.f;
  }
}

// ---------------------------------------------------------------------------------------------
// One-exponential step (direct modes, M <= kOnceMaxM traps).  The back-projection and the
// forward field of an iteration use the same pair exponentials E_j^m = e^{i Delta_j^m}:
//   S_j = sum_m c_m E_j^m,  c_m = w_m V_m/|V_m|      (back-projection, Sec. 3)
//   u_j = e^{i arg S_j}                              (the new phase, phi_j = arg S_j)
//   N V_m = sum_j u_j conj(E_j^m)                    (forward field, Eq. 1).
// A thread keeps the exponentials of its pixels and traps in registers between the two sums,
// so each pair costs one cos/sin per iteration instead of two.  The 8 warps of a block split
// the traps (warp_traps over all M, at most TMAX each, fixed for the launch); lane l holds
// column x0 + l of a sub-tile of at most R rows.  All M traps' tables of a sub-tile are staged
// in shared memory at once (the column parts once per 32-pixel strip), one sub-tile ahead.  A
// thread's forward sums stay in registers over all of the block's sub-tiles; they are summed
// over the warp and added, in fixed point, once at the end.  The forward-only variant (the
// field of given phases) evaluates the same expressions in the same order, so a sequence
// resumed from stored phases gives the same bits.
constexpr int kOnceMaxM = 128;
constexpr int kOnceTMax = 16;  // traps per warp at most (8 warps x 16 = kOnceMaxM)
// Rows per sub-tile of the forward field of given phases (no exponentials kept between sub-tiles,
// so taller sub-tiles: fewer barriers).  Its block runs are the step's, cut into sub-tiles of
// these rows: per trap the same rows are added in the same order, so the sums are the bits of
// the step's forward field.
constexpr int kOnceFwdRows = 8;

// Floats per trap in a staged block of row parts (R rows, in 16-byte pieces).
__host__ __device__ constexpr int once_yw(int R) { return (R + 3) & ~3; }

// Shared memory of a block: the coefficients, the row parts of two sub-tiles and the column
// parts of two strips (the next ones are staged during the current sub-tile), the warps'
// partial superpositions and the unit phasors u_j.
__host__ __device__ constexpr int once_smem_bytes(int R) {
  return kOnceMaxM * 8 + kWarps * kOnceTMax * 8 + 2 * kOnceMaxM * once_yw(R) * 4 + 2 * kOnceMaxM * kTileW * 4 +
         kWarps * R * kTileW * 8 + R * kTileW * 8;
}

struct OnceSmem {
  float2 *C;   // [kOnceMaxM] complex coefficients (gsw_prologue<true>)
  float2 *Cw;  // [kWarps][kOnceTMax] each warp's coefficients, zero past its traps
  float *Yb;   // [2][kOnceMaxM][once_yw(R)] row parts of a sub-tile's rows, by trap
  float *Xb;   // [2][kOnceMaxM][kTileW] column parts of a strip, by trap
  float2 *Sp;  // [kWarps][R][kTileW] per-warp superpositions
  float2 *Ps;  // [R][kTileW] unit phasors of the sub-tile's pixels (0 outside the image)
  int yw;
  __device__ __forceinline__ OnceSmem(unsigned char *raw, int R) {
    yw = once_yw(R);
    C = reinterpret_cast<float2 *>(raw);
    Cw = C + kOnceMaxM;
    Yb = reinterpret_cast<float *>(Cw + kWarps * kOnceTMax);
    Xb = Yb + 2 * kOnceMaxM * yw;
    Sp = reinterpret_cast<float2 *>(Xb + 2 * kOnceMaxM * kTileW);
    Ps = Sp + kWarps * R * kTileW;
  }
  __device__ __forceinline__ float *rows(int buf) const { return Yb + buf * kOnceMaxM * yw; }
  __device__ __forceinline__ float *cols(int buf) const { return Xb + buf * kOnceMaxM * kTileW; }
};

// Issues the asynchronous copies of the column parts X_m(x0 .. x0 + 31) of every trap into Xb
// (16-byte pieces when the strip lies inside the image and W is a multiple of 4; zero past the
// right edge otherwise).  Not committed.
__device__ __forceinline__ void once_stage_columns(const StepArgs &a, int x0, float *Xb) {
  if ((a.W & 3) == 0 && x0 + kTileW <= a.W) {
    for (int i = gthread(); i < a.M * (kTileW / 4); i += kThreads) {
      const int k = i >> 3, q = i & 7;
      cp_async16(Xb + k * kTileW + 4 * q, a.X + (size_t)k * a.W + x0 + 4 * q);
    }
  } else {
    for (int i = gthread(); i < a.M * kTileW; i += kThreads) {
      const int k = i / kTileW, col = x0 + (i % kTileW);
      const bool ok = col < a.W;
      cp_async4(Xb + i, a.X + (ok ? (size_t)k * a.W + col : 0), ok);
    }
  }
}

// Issues the asynchronous copies of the row parts Y_m(y0 .. y0 + R - 1) of every trap into Yb
// (once_yw(R) floats per trap, 16-byte pieces of the aligned shifted copy when there is one).
// Not committed.
template <int R>
__device__ __forceinline__ void once_stage_rows(const StepArgs &a, const SubTile &st, float *Yb) {
  constexpr int YW = once_yw(R), Q = YW / 4;
  if (a.Y4) {
    const int s = (4 - (st.y0 & 3)) & 3;
    const float *src = a.Y4 + (size_t)s * a.M * a.ldy4 + st.y0 + s;
    for (int i = gthread(); i < a.M * Q; i += kThreads) {
      const int k = i / Q, q = i % Q;
      cp_async16(Yb + k * YW + 4 * q, src + (size_t)k * a.ldy4 + 4 * q);
    }
  } else {
    for (int i = gthread(); i < a.M * YW; i += kThreads) {
      const int k = i / YW, r = i % YW;
      const bool ok = r < st.rows;
      cp_async4(Yb + i, a.Y + (ok ? (size_t)k * a.H + st.y0 + r : 0), ok);
    }
  }
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Two FP32 values in one 64-bit register for the packed FP32 instructions of sm_100 and later
// (add / fma .f32x2): one instruction does both lanes, each rounded as the scalar operation.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// u = e^{i phi} of a phase reduced to one turn in table units: radians in [-pi, pi] (fast,
// scaled by 1 + kFastEta here like the tables) or turns in [-1/2, 1/2] (accurate).
template <bool FAST>
__device__ __forceinline__ float2 unit_phasor(float ph) {
  float s, c;
  if (FAST) {
    const float x = fmaf(ph, kFastEta, ph);
    s = sin_approx(x);
    c = cos_approx(x);
  } else {
    sincospif(2.0f * ph, &s, &c);
  }
  return make_float2(c, s);
}

constexpr int kOnceLast = 1, kOnceReadU = 2;  // StepArgs::once_flags

// u = S/|S|, the unit phasor e^{i arg S} without the angle; 1 for S = 0 (atan2(0, 0) = 0).
__device__ __forceinline__ float2 unit_of(float2 s) {
  float q = abs2(s);
  if (q < 0x1p-100f) {  // |S| below 2^-50: scaled by 2^64 (exactly) so that |S|^2 stays a normal number
    s.x *= 0x1p64f;
    s.y *= 0x1p64f;
    q = abs2(s);
  }
  if (q == 0.f) return make_float2(1.f, 0.f);
  const float r = rsqrtf(q);
  return make_float2(s.x * r, s.y * r);
}

// Back-projection of a warp's TV traps (tables and coefficients from Xs, Yb, Cw, trap by trap)
// onto the lane's R rows: E[k][r] = e^{i (X + Y)} (kept), S[r] = sum_k c_k E[k][r], accumulated
// as U[r] = sum_k Re(c_k) E[k][r] and W[r] = sum_k Im(c_k) E[k][r] (S = U + i W) with packed FP32
// multiply-adds on E's (cos, sin) pair; the arguments X + Y of two rows are one packed add.  All
// R rows are evaluated (no per-row branches): the rows past a short sub-tile's end are staged
// rows of the next sub-tile or zero padding, and their results are discarded.
// PIPE: the forward field of the previous sub-tile is fused in -- each of its exponentials is
// used for acc[k] += Pp[r] conj(E[k][r]) just before it is replaced -- so that its FP32 work
// overlaps this sub-tile's cos/sin (per trap the rows and sub-tiles are added in the same order
// as by once_accumulate, so the sums are the same bits).
template <bool FAST, int TV, int R, bool PIPE>
__device__ __forceinline__ void once_back(const float *Xs, const float *Yb, const float2 *Cw, int lane,
                                          float2 (&E)[TV][R], float2 (&S)[R], const float2 (&Pp)[R],
                                          float2 (&acc)[TV]) {
  constexpr int YW = once_yw(R);
  unsigned long long U[R], Wp[R];
#pragma unroll
  for (int r = 0; r < R; r++) U[r] = Wp[r] = 0ull;  // (+0, +0)
#pragma unroll
  for (int k = 0; k < TV; k++) {
    const float2 c = Cw[k];
    const unsigned long long cx = pack2(c.x, c.x), cy = pack2(c.y, c.y);
    const float xk = Xs[k * kTileW + lane];
    const unsigned long long xx = pack2(xk, xk);
    const ulonglong2 *yq = reinterpret_cast<const ulonglong2 *>(Yb + k * YW);
#pragma unroll
    for (int h = 0; h < (R + 1) / 2; h++) {
      const ulonglong2 y4 = yq[h / 2];  // rows 4 (h / 2) .. + 3, one 16-byte load
      const float2 arg = unpack2(add2(xx, (h & 1) ? y4.y : y4.x));  // rows 2h and 2h + 1
      const float a2[2] = {arg.x, arg.y};
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const int r = 2 * h + j;
        if (r < R) {
          if (PIPE) {
            acc[k].x = fmaf(Pp[r].x, E[k][r].x, fmaf(Pp[r].y, E[k][r].y, acc[k].x));
            acc[k].y = fmaf(Pp[r].y, E[k][r].x, fmaf(-Pp[r].x, E[k][r].y, acc[k].y));
          }
          float co, si;
          cis<FAST>(a2[j], co, si);
          E[k][r] = make_float2(co, si);
          const unsigned long long e = pack2(co, si);
          U[r] = fma2(cx, e, U[r]);
          Wp[r] = fma2(cy, e, Wp[r]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; r++) {
    const float2 u = unpack2(U[r]), w = unpack2(Wp[r]);
    S[r] = make_float2(u.x - w.y, u.y + w.x);
  }
}

// acc[k] += u_r conj(E[k][r]) over the lane's R rows (u_r = 0 past the sub-tile's end).
template <int TV, int R>
__device__ __forceinline__ void once_accumulate(const float2 (&P)[R], const float2 (&E)[TV][R], float2 (&acc)[TV]) {
#pragma unroll
  for (int k = 0; k < TV; k++) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      acc[k].x = fmaf(P[r].x, E[k][r].x, fmaf(P[r].y, E[k][r].y, acc[k].x));
      acc[k].y = fmaf(P[r].y, E[k][r].x, fmaf(-P[r].x, E[k][r].y, acc[k].y));
    }
  }
}

// Forward field of given phases: the exponentials of the back-projection's expression, then the
// same accumulation (trap by trap, one trap's rows at a time).
template <bool FAST, int TV, int R>
__device__ __forceinline__ void once_forward_only(const float *Xs, const float *Yb, const float2 (&P)[R], int lane,
                                                  float2 (&acc)[TV]) {
  constexpr int YW = once_yw(R);
#pragma unroll
  for (int k = 0; k < TV; k++) {
    float2 E[1][R];
    const float xk = Xs[k * kTileW + lane];
    const float4 *yq = reinterpret_cast<const float4 *>(Yb + k * YW);
#pragma unroll
    for (int q = 0; q < YW / 4; q++) {
      const float4 y4 = yq[q];
      const float yy[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int r = 4 * q + j;
        if (r < R) cis<FAST>(xk + yy[j], E[0][r].x, E[0][r].y);
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      acc[k].x = fmaf(P[r].x, E[0][r].x, fmaf(P[r].y, E[0][r].y, acc[k].x));
      acc[k].y = fmaf(P[r].y, E[0][r].x, fmaf(-P[r].x, E[0][r].y, acc[k].y));
    }
  }
}

// The sub-tiles of a block, for a warp whose traps lo .. lo + T - 1 are evaluated as TV traps
// (T <= TV; the rest are padding: zero coefficients, their sums dropped), then the warp's
// forward sums, totalled over its lanes in a fixed order and added in fixed point.
// PIPE: the forward field of each sub-tile runs inside the next sub-tile's back-projection
// (once_back), the last one's after the loop.
// BACK: the forward field takes u_j = S_j/|S_j|; last: phi_j = atan2(S_j) is written (and u_j to
// a.u when set).  Otherwise u_j is read from a.u under kOnceReadU, else e^{i phi_j} from a.phi.
template <bool FAST, bool BACK, int TV, int R, bool PIPE>
__device__ __forceinline__ void once_loop(const StepArgs &a, const OnceSmem &sm, int t_begin, int t_end, int lo,
                                          int T, bool last) {
  const int lane = threadIdx.x & 31, warp = gthread() >> 5, t = gthread();
  constexpr int YW = once_yw(R);
  float2 acc[TV];
#pragma unroll
  for (int k = 0; k < TV; k++) acc[k] = make_float2(0.f, 0.f);
  // the sub-tile's exponentials and unit phasors (PIPE: the previous sub-tile's until replaced;
  // zero before the first, which adds nothing)
  float2 E[TV][R], P[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    P[r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < TV; k++) E[k][r] = make_float2(0.f, 0.f);
  }
  int xb = 0;  // the buffer of the current strip's column parts
  for (int i = t_begin; i < t_end; i++) {
    const SubTile st = a.sub[i];
    const int buf = (i - t_begin) & 1;
    if (!BACK) group_sync();  // the previous sub-tile's readers of Ps and of the other buffers are done
    bool next_strip = false;
    if (i + 1 < t_end) {  // stage the next sub-tile's tables
      const SubTile nx = a.sub[i + 1];
      once_stage_rows<R>(a, nx, sm.rows(buf ^ 1));
      next_strip = nx.x0 != st.x0;
      if (next_strip) once_stage_columns(a, nx.x0, sm.cols(xb ^ 1));
    }
    cp_async_commit();  // (an empty group after the last sub-tile: uniform waits)
    const float *Xs = sm.cols(xb) + lo * kTileW, *Yb = sm.rows(buf) + lo * YW;
    if (BACK) {
      float2 S[R];
#pragma unroll
      for (int r = 0; r < R; r++) S[r] = make_float2(0.f, 0.f);
      once_back<FAST, TV, R, PIPE>(Xs, Yb, sm.Cw + warp * kOnceTMax, lane, E, S, P, acc);
#pragma unroll
      for (int r = 0; r < R; r++)
        if (r < st.rows) sm.Sp[(warp * R + r) * kTileW + lane] = S[r];
      group_sync();
      if (t < st.rows * kTileW) {  // one pixel per thread: the 8 warps' sums in warp order
        const int r = t >> 5, l = t & 31, ix = st.x0 + l;
        float2 s = sm.Sp[r * kTileW + l];
#pragma unroll
        for (int w = 1; w < kWarps; w++) {
          const float2 q = sm.Sp[(w * R + r) * kTileW + l];
          s.x += q.x;
          s.y += q.y;
        }
        const float2 u = unit_of(s);
        if (last && ix < a.W) {
          const size_t j = (size_t)(st.y0 + r) * a.W + ix;
          a.phi[j] = atan2f(s.y, s.x);
          if (a.u) a.u[j] = u;
        }
        sm.Ps[r * kTileW + l] = ix < a.W ? u : make_float2(0.f, 0.f);
      }
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // the next sub-tile's tables
    } else {
      if (t < st.rows * kTileW) {
        const int r = t >> 5, l = t & 31, ix = st.x0 + l;
        const size_t j = (size_t)(st.y0 + r) * a.W + ix;
        float2 u = make_float2(0.f, 0.f);
        if (ix < a.W)
          u = (a.once_flags & kOnceReadU) ? a.u[j]
                                          : unit_phasor<FAST>(FAST ? reduced_radians(a.phi[j]) : reduced_phase_turns(a.phi[j]));
        sm.Ps[r * kTileW + l] = u;
      }
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // this sub-tile's tables
    }
    group_sync();
#pragma unroll
    for (int r = 0; r < R; r++) P[r] = r < st.rows ? sm.Ps[r * kTileW + lane] : make_float2(0.f, 0.f);
    if (!BACK)
      once_forward_only<FAST, TV, R>(Xs, Yb, P, lane, acc);
    else if (!PIPE)
      once_accumulate<TV, R>(P, E, acc);
    if (next_strip) xb ^= 1;
  }
  if (BACK && PIPE) once_accumulate<TV, R>(P, E, acc);  // the forward field of the last sub-tile
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  unsigned long long *const out = block_acc(a);
#pragma unroll
  for (int g = 0; g < TV; g += kGroup) {
    float2 v8[kGroup];
#pragma unroll
    for (int i = 0; i < kGroup; i++) v8[i] = g + i < TV ? acc[g + i] : make_float2(0.f, 0.f);
    const float2 v = warp_reduce8(v8, lane);
    const int k = g + ((lane >> 2) & 7);
    if ((lane & 3) == 0 && k < T) {
      // |v| <= the block's pixel count <= N, so v * 2^fx_shift is an exact integer below 2^62
      atomicAdd(out + lo + k, (unsigned long long)__float2ll_rn(v.x * a.fx_scale));
      atomicAdd(out + a.M + lo + k, (unsigned long long)__float2ll_rn(v.y * a.fx_scale));
    }
  }
}

// The work of one block on its sub-tiles [t_begin, t_end) after the dependency wait and the
// clearing of the next accumulator.  On entry the first sub-tile's row and column parts are
// being staged into rows(0) and cols(0) (one committed group).
// BACK: weight update, back-projection -> a.phi, forward field of the new phases; otherwise
// the forward field of the phases in a.phi.
// A warp's trap count T is TMAX, TMAX - 1 or TMAX - 2 (warp_traps); every warp runs the loop
// compiled for TMAX traps, the ones past T as padding, so that no per-trap branch remains and
// one copy of the unrolled loop serves the block (with the fused forward field, copies for T
// and T - 1 ran slower).  From 4 traps per warp, with at most 32 exponentials per thread, each
// sub-tile's forward field is fused into the next sub-tile's back-projection (with more the
// registers spill; with 2 traps per warp it does not pay).
template <bool FAST, bool BACK, int TMAX, int R>
__device__ __forceinline__ void once_block(const StepArgs &a, const OnceSmem &sm, int t_begin, int t_end,
                                           float *trace, bool last) {
  static_assert(TMAX >= 1 && TMAX <= kOnceTMax, "traps per warp");
  const int lane = threadIdx.x & 31, warp = gthread() >> 5;
  int lo, hi;
  warp_traps(a.M, warp, lo, hi);
  const int T = hi - lo;
  if (BACK) {  // the weights are written here, before the sub-tiles: nothing stays live across them
    LateWeight lw;
    gsw_prologue<true>(a, a.M, sm.C, vblock(), vgrid(), lw, trace);
    write_weights<true>(a, lw, vgrid());
  }
  // Padding traps read table rows from M on (never staged): zero, in both buffers.
  for (int i = gthread(); i < 2 * kOnceTMax * (kTileW + sm.yw); i += kThreads) {
    const int b = i / (kOnceTMax * (kTileW + sm.yw)), j = i % (kOnceTMax * (kTileW + sm.yw));
    if (j < kOnceTMax * kTileW) {
      if (a.M * kTileW + j < kOnceMaxM * kTileW) sm.cols(b)[a.M * kTileW + j] = 0.f;
    } else if (a.M * sm.yw + (j - kOnceTMax * kTileW) < kOnceMaxM * sm.yw) {
      sm.rows(b)[a.M * sm.yw + (j - kOnceTMax * kTileW)] = 0.f;
    }
  }
  if (BACK) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    group_sync();  // coefficients, padding and the first tables are in place
    if (lane < kOnceTMax) sm.Cw[warp * kOnceTMax + lane] = lane < T ? sm.C[lo + lane] : make_float2(0.f, 0.f);
    __syncwarp();
  }
  constexpr bool PIPE = TMAX >= 4 && TMAX * R <= 32;
  once_loop<FAST, BACK, TMAX, R, PIPE>(a, sm, t_begin, t_end, lo, T, last);
}

// Stages the first sub-tile's tables of a block (one committed group; empty without work).
template <int R>
__device__ __forceinline__ void once_stage_first(const StepArgs &a, const OnceSmem &sm, int t_begin, int t_end) {
  if (t_begin < t_end) {
    const SubTile st0 = a.sub[t_begin];
    once_stage_rows<R>(a, st0, sm.rows(0));
    once_stage_columns(a, st0.x0, sm.cols(0));
  }
  cp_async_commit();
}

// The shape of M traps (0: none, M > kOnceMaxM): TMAX = ceil(M / 8) traps per warp at most.
__host__ __device__ constexpr int once_shape(int M) { return M <= 0 || M > kOnceMaxM ? 0 : (M + kWarps - 1) / kWarps; }
// R, the rows per sub-tile of a shape: 8 up to 4 traps per warp, 3 for 11 (faster there than 2),
// otherwise the largest R with TMAX R <= 32 (the fused forward field, once_block).
__host__ __device__ constexpr int once_rows(int shape) {
  return shape <= 4 ? 8 : shape == 11 ? 3 : 32 / shape < 8 ? 32 / shape : 8;
}

// Calls BODY (parenthesised) with compile-time TMAX and R of a shape (once_shape).
#define HOT_ONCE_CASE(k, BODY) \
  case k: { constexpr int TMAX = k, R = ::hot::once_rows(k); BODY; } break;
#define HOT_WITH_ONCE_SHAPE(shape, BODY)                                                        \
  switch (shape) {                                                                              \
    HOT_ONCE_CASE(1, BODY) HOT_ONCE_CASE(2, BODY) HOT_ONCE_CASE(3, BODY) HOT_ONCE_CASE(4, BODY)   \
    HOT_ONCE_CASE(5, BODY) HOT_ONCE_CASE(6, BODY) HOT_ONCE_CASE(7, BODY) HOT_ONCE_CASE(8, BODY)   \
    HOT_ONCE_CASE(9, BODY) HOT_ONCE_CASE(10, BODY) HOT_ONCE_CASE(11, BODY) HOT_ONCE_CASE(12, BODY) \
    HOT_ONCE_CASE(13, BODY) HOT_ONCE_CASE(14, BODY) HOT_ONCE_CASE(15, BODY)                      \
    default: HOT_ONCE_CASE(16, BODY)                                                            \
  }

// The per-launch form.  The tables are constant during hot_gsw: the first sub-tile's are
// staged before waiting for the previous launch.
template <bool FAST, bool BACK, int TMAX, int R>
__global__ void __launch_bounds__(kThreads, 2) gsw_once_kernel(StepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const OnceSmem sm(smem_raw, R);
  const int vb = vblock(), vg = vgrid();
  const int t_begin = a.first[vb], t_end = a.first[vb + 1];
  allow_dependents();
  once_stage_first<R>(a, sm, t_begin, t_end);
  grid_dependency_wait();
  for (int i = vb * kThreads + gthread(); i < 2 * a.M * a.copies; i += vg * kThreads) a.acc_clear[i] = 0ull;
  once_block<FAST, BACK, TMAX, R>(a, sm, t_begin, t_end, a.trace, (a.once_flags & kOnceLast) != 0);
}

// ---------------------------------------------------------------------------------------------
// Separable variant.  Eq. 2 is a sum of a column part and a row part, so every pair's
// exponential factorises: e^{i Delta_j^m} = Xc_m(ix) Yc_m(iy), with both factors tabulated once
// per trap (FP64 cos/sin of the exactly reduced turns, stored as FP32 complex).  Per pair the
// back-projection then takes one complex multiply-add,
//   S_j += Yc_m(iy) [c_m Xc_m(ix)]           (the bracket once per trap and lane),
// and the forward field another,
//   V_m += conj(Xc_m(ix)) sum_iy u_j conj(Yc_m(iy))   with u_j = e^{i phi_j},
// i.e. 8 FP32 FMA per pixel-trap update and no per-pair transcendental function (one sincos
// per pixel and iteration gives u_j from the stored phase).  The coefficients are kept
// complex, c_m = w_m V_m/|V_m| (Sec. 3).
// The work decomposition, staging, reductions and fixed-point sums are the direct kernel's.
constexpr int kSepUsFloats = kRowsMax * kTileW * 2;

__host__ __device__ constexpr int sep_smem_bytes(int chunk) {
  return chunk * (kTileW + kYStride) * 8 + 2 * chunk * 8 + kWarps * kHalfRows * kTileW * 8 + kSepUsFloats * 4;
}

struct SepSmem {
  float2 *Xs, *Ys, *Cs, *Sp, *Us, *C0;
  __device__ __forceinline__ SepSmem(unsigned char *raw, int chunk) {
    Xs = reinterpret_cast<float2 *>(raw);  // [chunk][kTileW]
    Ys = Xs + chunk * kTileW;              // [chunk][kYStride]
    Cs = Ys + chunk * kYStride;            // [chunk]
    Sp = Cs + chunk;                       // [kWarps][kHalfRows][kTileW]
    Us = Sp + kWarps * kHalfRows * kTileW; // [kRowsMax][kTileW] unit phasors of the sub-tile
    C0 = Us + kRowsMax * kTileW;           // [chunk] coefficients of the first chunk (prologue)
  }
};

// Sec. 3 coefficient of trap m in complex form: w_m' V_m/|V_m| with w_m' = w_m <|V|>/|V_m|
// (R4: |V_m| = 0 keeps w_m and takes the unit field 1).
__device__ __forceinline__ float2 complex_coefficient(const StepArgs &a, int m, float mean) {
  return update_from<true>(field_from_sums<true>(a, m), __ldcg(a.w_in + m), mean, 1.f);
}

template <bool BACK, bool ADJ = false>
__device__ __forceinline__ void stage_sep(const StepArgs &a, int m0, int n, const SubTile &st, const SepSmem &sm,
                                          bool xy = true, float mean = 0.f, bool coef = true) {
  if (xy) {
    if ((a.W & 1) == 0 && st.x0 + kTileW <= a.W) {
      // thread t copies columns 2 (t % 16), +1 of traps t / 16, t / 16 + 16, ... (16 bytes:
      // rows start 16-byte aligned for even W)
      const int q = gthread() % (kTileW / 2), kx = gthread() / (kTileW / 2);
      const float2 *src = a.Xc + (size_t)(m0 + kx) * a.W + st.x0 + 2 * q;
      const size_t sx = (size_t)(kThreads / (kTileW / 2)) * a.W;
      for (int k = kx; k < n; k += kThreads / (kTileW / 2), src += sx) cp_async16(sm.Xs + k * kTileW + 2 * q, src);
    } else {
      // thread t copies column t % 32 of traps t / 32, t / 32 + 8, ...: fixed column, pointers
      // advanced by whole trap strides
      const int col = gthread() % kTileW, kx = gthread() / kTileW;
      const bool okx = st.x0 + col < a.W;
      const float2 *src = a.Xc + (okx ? (size_t)(m0 + kx) * a.W + st.x0 + col : 0);
      const size_t sx = okx ? (size_t)(kThreads / kTileW) * a.W : 0;
      for (int k = kx; k < n; k += kThreads / kTileW, src += sx) cp_async8(sm.Xs + k * kTileW + col, src, okx);
    }
    // rows y0 .. y0 + 15 of copy y0 % 2 (16-byte aligned): thread t copies rows 2 (t % 8), +1 of
    // traps t / 8, t / 8 + 32, ...
    const int s = st.y0 & 1, q = gthread() % (kYStride / 2), ky = gthread() / (kYStride / 2);
    const float2 *srcy = a.Yc + ((size_t)s * a.M + m0 + ky) * a.ldy4 + st.y0 + s + 2 * q;
    const size_t sy = (size_t)(kThreads / (kYStride / 2)) * a.ldy4;
    for (int k = ky; k < n; k += kThreads / (kYStride / 2), srcy += sy) cp_async16(sm.Ys + k * kYStride + 2 * q, srcy);
  }
  if (BACK && coef)
    for (int i = gthread(); i < n; i += kThreads)
      sm.Cs[i] = (ADJ || a.G) ? a.G[m0 + i] : complex_coefficient(a, m0 + i, mean);
  cp_async_wait_all();
}

// S_r += Yc_m(r) (c_m Xc_m(lane)) for traps [lo, hi) of the staged chunk (coefficients C).
template <int R>
__device__ __forceinline__ void back_traps_sep(const SepSmem &sm, const float2 *C, int lo, int hi, int lane,
                                               float2 (&S)[kRowsMax]) {
  for (int k = lo; k < hi; k++) {
    const float2 x = sm.Xs[k * kTileW + lane], c = C[k];
    const float2 b = make_float2(c.x * x.x - c.y * x.y, c.x * x.y + c.y * x.x);
    const float4 *yq = reinterpret_cast<const float4 *>(sm.Ys + k * kYStride);
#pragma unroll
    for (int q = 0; q < (R + 1) / 2; q++) {
      const float4 y2 = yq[q];
      const float2 yy[2] = {make_float2(y2.x, y2.y), make_float2(y2.z, y2.w)};
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const int r = 2 * q + j;
        if (r < R) {
          S[r].x = fmaf(yy[j].x, b.x, fmaf(-yy[j].y, b.y, S[r].x));
          S[r].y = fmaf(yy[j].x, b.y, fmaf(yy[j].y, b.x, S[r].y));
        }
      }
    }
  }
}

// Forward field of traps [lo, hi): conj(Xc_m(lane)) sum_r u_r conj(Yc_m(r)), summed over the
// warp 8 traps at a time and added in fixed point (as forward_traps).  u is zero outside the
// image, so no mask is needed.
template <int R>
__device__ __forceinline__ void forward_traps_sep(const SepSmem &sm, int lo, int hi, int lane,
                                                  const float2 (&u)[kRowsMax], const StepArgs &a, int m0) {
  for (int g = lo; g < hi; g += kGroup) {
    float2 acc[kGroup];
#pragma unroll
    for (int i = 0; i < kGroup; i++) {
      acc[i] = make_float2(0.f, 0.f);
      const int k = g + i;
      if (k < hi) {
        const float4 *yq = reinterpret_cast<const float4 *>(sm.Ys + k * kYStride);
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < (R + 1) / 2; q++) {
          const float4 y2 = yq[q];
          const float2 yy[2] = {make_float2(y2.x, y2.y), make_float2(y2.z, y2.w)};
#pragma unroll
          for (int j = 0; j < 2; j++) {
            const int r = 2 * q + j;
            if (r < R) {
              t.x = fmaf(u[r].x, yy[j].x, fmaf(u[r].y, yy[j].y, t.x));
              t.y = fmaf(u[r].y, yy[j].x, fmaf(-u[r].x, yy[j].y, t.y));
            }
          }
        }
        const float2 x = sm.Xs[k * kTileW + lane];
        acc[i] = make_float2(t.x * x.x + t.y * x.y, t.y * x.x - t.x * x.y);
      }
    }
    const float2 v = warp_reduce8(acc, lane);
    const int k = g + ((lane >> 2) & 7);
    if ((lane & 3) == 0 && k < hi) {
      unsigned long long *acc = block_acc(a);
      atomicAdd(acc + m0 + k, (unsigned long long)__float2ll_rn(v.x * a.fx_scale));
      atomicAdd(acc + a.M + m0 + k, (unsigned long long)__float2ll_rn(v.y * a.fx_scale));
    }
  }
}

template <bool BACK, bool FWD, bool ADJ>
__device__ __forceinline__ void process_subtile_sep(const StepArgs &a, const SubTile st, float mean, bool &prestaged,
                                                    const SepSmem &sm, const float2 *C0 = nullptr) {
  const int lane = threadIdx.x & 31, warp = gthread() >> 5;
  const int mc = a.M < a.chunk ? a.M : a.chunk;
  const int nchunks = (a.M + mc - 1) / mc;
  const int ix = st.x0 + lane;
  const bool col_ok = ix < a.W;

  if (BACK) {
    float2 S[kRowsMax];
#pragma unroll
    for (int r = 0; r < kRowsMax; r++) S[r] = make_float2(0.f, 0.f);
    for (int ch = 0; ch < nchunks; ch++) {
      const int m0 = ch * mc, n = min(mc, a.M - m0);
      const bool pre = C0 && ch == 0;
      group_sync();  // earlier readers of the tables are done
      stage_sep<true, ADJ>(a, m0, n, st, sm, !prestaged, mean, !pre);
      prestaged = false;
      group_sync();
      int lo, hi;
      warp_traps(n, warp, lo, hi);
      const float2 *C = pre ? C0 : sm.Cs;
      HOT_WITH_ROWS(st.rows, (back_traps_sep<R>(sm, C, lo, hi, lane, S)));
    }
#pragma unroll
    for (int h = 0; h < 2; h++) {
      if (h * kHalfRows >= st.rows) break;
      group_sync();  // Sp and the phasor rows are free
#pragma unroll
      for (int i = 0; i < kHalfRows; i++)
        if (h * kHalfRows + i < st.rows) sm.Sp[(warp * kHalfRows + i) * kTileW + lane] = S[h * kHalfRows + i];
      group_sync();
      if (warp < kHalfRows && h * kHalfRows + warp < st.rows) {
        const int r = h * kHalfRows + warp;
        float2 s = sm.Sp[warp * kTileW + lane];
#pragma unroll
        for (int w = 1; w < kWarps; w++) {
          const float2 q = sm.Sp[(w * kHalfRows + warp) * kTileW + lane];
          s.x += q.x;
          s.y += q.y;
        }
        const size_t j = (size_t)(st.y0 + r) * a.W + ix;
        if (ADJ) {
          if (col_ok) {
            float sp, cp;
            sincosf(a.phi[j], &sp, &cp);
            a.grad[j] = (cp * s.y - sp * s.x) * a.inv_n;  // Im[(cos - i sin)(S.x + i S.y)] / N
          }
        } else {
          const float ph = atan2f(s.y, s.x);
          if (col_ok) a.phi[j] = ph;
          if (FWD) {  // u = e^{i phi} of the stored phase (so that a resumed run is identical)
            float2 u = make_float2(0.f, 0.f);
            if (col_ok) sincosf(ph, &u.y, &u.x);
            sm.Us[r * kTileW + lane] = u;
          }
        }
      }
    }
  } else if (FWD) {
    group_sync();  // earlier readers of the phasors and of the tables are done
    for (int r = warp; r < st.rows; r += kWarps) {
      float2 u = make_float2(0.f, 0.f);
      if (col_ok) sincosf(a.phi[(size_t)(st.y0 + r) * a.W + ix], &u.y, &u.x);
      sm.Us[r * kTileW + lane] = u;
    }
  }

  if (FWD) {
    group_sync();  // the phasors are complete
    float2 u[kRowsMax];
#pragma unroll
    for (int r = 0; r < kRowsMax; r++) u[r] = r < st.rows ? sm.Us[r * kTileW + lane] : make_float2(0.f, 0.f);
    for (int ch = 0; ch < nchunks; ch++) {
      const int m0 = ch * mc, n = min(mc, a.M - m0);
      if (!BACK || nchunks > 1) {  // with one chunk the back-projection's tables are still staged
        if (ch) group_sync();
        stage_sep<false>(a, m0, n, st, sm);
        group_sync();
      }
      int lo, hi;
      warp_traps(n, warp, lo, hi);
      HOT_WITH_ROWS(st.rows, (forward_traps_sep<R>(sm, lo, hi, lane, u, a, m0)));
    }
  }
}

template <bool BACK, bool FWD, bool ADJ = false>
// Two resident blocks per SM: the complex accumulators and tables of the separable loops need
// more than the 80 registers of three blocks (measured 15 % faster at 512^2, M = 100).
__global__ void __launch_bounds__(kThreads, 2) gsw_sep_kernel(StepArgs a) {
  static_assert(!ADJ || (BACK && !FWD), "the adjoint is a back-projection without forward field");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SepSmem sm(smem_raw, a.chunk);
  const int mc = a.M < a.chunk ? a.M : a.chunk;
  const int t_begin = a.first[blockIdx.x], t_end = a.first[blockIdx.x + 1];

  allow_dependents();
  bool prestaged = false;
  if (BACK && t_begin < t_end) {
    stage_sep<false>(a, 0, mc, a.sub[t_begin], sm);
    prestaged = true;
  }
  grid_dependency_wait();
  if (FWD)
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < 2 * a.M * a.copies; i += gridDim.x * kThreads) a.acc_clear[i] = 0ull;
  LateWeight lw;
  const bool gsw = BACK && !ADJ && !a.G;
  if (gsw) gsw_prologue<true>(a, mc, sm.C0, blockIdx.x, gridDim.x, lw, a.trace);
  for (int t = t_begin; t < t_end; t++)
    process_subtile_sep<BACK, FWD, ADJ>(a, a.sub[t], 1.f, prestaged, sm, gsw ? sm.C0 : nullptr);
  if (gsw) write_weights<true>(a, lw, gridDim.x);
}

// Batched launch: the sub-tiles of up to kBatchMax holograms (SubTile::pad = hologram index)
// in one grid.  The holograms' parameters travel in the launch itself (a __grid_constant__
// argument read through the constant cache, as the single-hologram kernel reads its own).
// Every block that meets a hologram computes its <|V|> and coefficients itself; the weights
// of hologram h are written by block owner[h].
constexpr int kBatchMax = 22;  // keeps the launch argument under 4 KB

struct BatchArgs {
  StepArgs holo[kBatchMax];
  int owner[kBatchMax];
  const SubTile *sub;
  const int *first;  // [gridDim.x + 1]
  int count;
};
static_assert(sizeof(BatchArgs) <= 4096, "launch argument above 4 KB");

// MODE: kModeAccurate, kModeFast or kModeSeparable (the separable kernel's staging capacity is
// the batch's chunk, the same for all holograms of a launch).
template <int MODE, bool BACK, bool FWD>
__global__ void __launch_bounds__(kThreads, MODE == kModeSeparable ? 2 : 4)
    gsw_batch_kernel(const __grid_constant__ BatchArgs b) {
  constexpr bool FAST = MODE == kModeFast, SEP = MODE == kModeSeparable;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t_begin = b.first[blockIdx.x], t_end = b.first[blockIdx.x + 1];
  const int cap = b.holo[0].chunk;
  float2 *const C0 = SEP ? SepSmem(smem_raw, cap).C0 : StepSmem(smem_raw).C0;

  allow_dependents();
  bool prestaged = false;
  if (BACK && t_begin < t_end) {
    const SubTile st0 = b.sub[t_begin];
    const StepArgs &a0 = b.holo[st0.pad];
    const int mc0 = a0.M < a0.chunk ? a0.M : a0.chunk;
    if constexpr (SEP) {
      stage_sep<false>(a0, 0, mc0, st0, SepSmem(smem_raw, cap));
    } else {
      const StepSmem sm(smem_raw);
      stage_tables<false>(a0, 0, mc0, st0, sm.Xs, sm.Ys, sm.Cs);
    }
    prestaged = true;
  }
  grid_dependency_wait();
  if (FWD)  // clear the buffers the next launch accumulates into, for every hologram
    for (int h = 0; h < b.count; h++) {
      unsigned long long *clr = b.holo[h].acc_clear;
      const int n2 = 2 * b.holo[h].M * b.holo[h].copies;
      for (int i = blockIdx.x * kThreads + threadIdx.x; i < n2; i += gridDim.x * kThreads) clr[i] = 0ull;
    }
  int cur = -1;
  LateWeight lw;  // the owner block writes all weights of a hologram, after its sub-tiles
  for (int t = t_begin; t < t_end; t++) {
    const SubTile st = b.sub[t];
    const StepArgs &a = b.holo[st.pad];
    if (BACK && st.pad != cur) {
      if (cur >= 0) write_weights<SEP>(b.holo[cur], lw, 1);
      const int mc = a.M < a.chunk ? a.M : a.chunk;
      gsw_prologue<SEP>(a, mc, C0, b.owner[st.pad] == (int)blockIdx.x ? 0 : a.M, 1, lw);
    }
    cur = st.pad;
    if constexpr (SEP)
      process_subtile_sep<BACK, FWD, false>(a, st, 1.f, prestaged, SepSmem(smem_raw, cap), BACK ? C0 : nullptr);
    else
      process_subtile<FAST, BACK, FWD, false>(a, st, 1.f, prestaged, StepSmem(smem_raw), BACK ? C0 : nullptr);
  }
  if (BACK && cur >= 0) write_weights<SEP>(b.holo[cur], lw, 1);
}

// ---------------------------------------------------------------------------------------------
// Persistent form: all launches of a hot_gsw call (the forward field of the starting phases and
// iterations 1..K) in one cooperative launch whose blocks are all resident, separated by a
// grid-wide barrier instead of kernel boundaries.  The arithmetic, the schedule and the
// fixed-point sums are those of the per-iteration kernels, so the results are the same bits.
// A block that owns a single sub-tile and a single trap chunk keeps that sub-tile's trap tables
// in shared memory for the whole call; only the coefficients are staged per iteration.

// Grid-wide barrier with a bounded wait.  count: arrivals since the launch began (zeroed
// before each launch; barrier j is passed when it reaches j x gridDim.x); err: set to 1 when a
// wait runs out (after limit_ns of %globaltimer), after which every block leaves at its next
// barrier and the host reports HOT_ETIMEOUT.
struct GridSync {
  unsigned int *count;
  int *err;
  long long limit_ns;
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_s32(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Every block calls this the same number of times.  epoch (thread 0's copy) is the arrival
// count that ends the previous barrier.  Returns false in every thread of the block if a wait
// ran out.
__device__ __forceinline__ bool grid_sync(const GridSync &g, unsigned int &epoch) {
  __shared__ int ok;
  __syncthreads();  // the block's writes and atomics of this phase are issued
  if (threadIdx.x == 0) {
    int good = 1;
    __threadfence();  // ordered after the block's writes by the barrier above
    epoch += gridDim.x;
    atomicAdd(g.count, 1u);
    const long long t0 = (long long)global_timer_ns();
    while (ld_acquire_u32(g.count) < epoch) {
      if (ld_acquire_s32(g.err)) {
        good = 0;
        break;
      }
      if ((long long)global_timer_ns() - t0 > g.limit_ns) {
        atomicExch(g.err, 1);
        good = 0;
        break;
      }
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// Parameters of the persistent kernels: launch k of the sequence uses step[k % 6] (the
// accumulators rotate over three buffers and the weights over two, as in hot_gsw).
struct PersistArgs {
  StepArgs step[6];
  int iters;
  int k0;  // one-exponential form: the first launch it runs (1: launch 0 was its own launch before it)
  GridSync sync;
  float *trace;  // NULL, or [iters][2]: e, u of the field read by iteration k (convergence trace)
};

template <int MODE>
__global__ void __launch_bounds__(kThreads, MODE == kModeSeparable ? 2 : 4)
    gsw_persistent_kernel(const __grid_constant__ PersistArgs p) {
  constexpr bool FAST = MODE == kModeFast;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const StepArgs &a0 = p.step[0];
  const int mc = a0.M < a0.chunk ? a0.M : a0.chunk;
  const int t_begin = a0.first[blockIdx.x], t_end = a0.first[blockIdx.x + 1];
  const bool resident = t_end - t_begin == 1 && a0.M <= a0.chunk;  // tables stay in shared memory
  unsigned int epoch = 0u;

  for (int k = 0; k <= p.iters; k++) {
    const StepArgs &a = p.step[k % 6];
    if (k > 0 && !grid_sync(p.sync, epoch)) return;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < 2 * a.M * a.copies; i += gridDim.x * kThreads) a.acc_clear[i] = 0ull;
    const float mean = 1.f;  // coefficients without the common factor <|V|> (see gsw_prologue)
    LateWeight lw;
    if constexpr (MODE == kModeSeparable) {
      const SepSmem sm(smem_raw, mc);
      if (k > 0) gsw_prologue<true>(a, mc, sm.C0, blockIdx.x, gridDim.x, lw, p.trace ? p.trace + 2 * (k - 1) : nullptr);
      for (int t = t_begin; t < t_end; t++) {
        bool prestaged = resident && k > 0;
        if (k == 0)
          process_subtile_sep<false, true, false>(a, a.sub[t], 0.f, prestaged, sm);
        else
          process_subtile_sep<true, true, false>(a, a.sub[t], mean, prestaged, sm, sm.C0);
      }
    } else {
      const StepSmem sm(smem_raw);
      if (k > 0) gsw_prologue<false>(a, mc, sm.C0, blockIdx.x, gridDim.x, lw, p.trace ? p.trace + 2 * (k - 1) : nullptr);
      for (int t = t_begin; t < t_end; t++) {
        bool prestaged = resident && k > 0;
        if (k == 0)
          process_subtile<FAST, false, true, false>(a, a.sub[t], 0.f, prestaged, sm);
        else
          process_subtile<FAST, true, true, false>(a, a.sub[t], mean, prestaged, sm, sm.C0);
      }
    }
    if (k > 0) write_weights<MODE == kModeSeparable>(a, lw, gridDim.x);
  }
}

// The persistent form of the one-exponential step (same schedule, same arithmetic, same bits).
template <bool FAST, int TMAX, int R>
__global__ void __launch_bounds__(kThreads, 2) gsw_once_persistent_kernel(const __grid_constant__ PersistArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const OnceSmem sm(smem_raw, R);
  const StepArgs &a0 = p.step[0];
  const int t_begin = a0.first[blockIdx.x], t_end = a0.first[blockIdx.x + 1];
  unsigned int epoch = 0u;
  for (int k = p.k0; k <= p.iters; k++) {
    const StepArgs &a = p.step[k % 6];
    if (k > p.k0 && !grid_sync(p.sync, epoch)) return;
    once_stage_first<R>(a, sm, t_begin, t_end);
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < 2 * a.M * a.copies; i += gridDim.x * kThreads) a.acc_clear[i] = 0ull;
    if (k == 0)
      once_block<FAST, false, TMAX, R>(a, sm, t_begin, t_end, nullptr, false);
    else
      once_block<FAST, true, TMAX, R>(a, sm, t_begin, t_end, p.trace ? p.trace + 2 * (k - 1) : nullptr, k == p.iters);
  }
}

// Per (trap, column) and (trap, row) phase parts of Eq. 2 reduced modulo one turn in FP64.
// abc: [M][3] = a_m, b_m, c_m in turns (see the file header).  Writes turns and radians.
// A row band (rows y_off .. y_off+H-1 of a hologram of H_total rows) takes the row parts of
// its global rows.
// Y4t, Y4r (optional): the shifted copies of the row parts (StepArgs::Y4), [4][M][ldy4], and
// Yc2 (optional) the two shifted copies of Yc (StepArgs::Yc), [2][M][ldy4], whose entries outside
// the shifted rows stay as they are (zero from allocation).
static __global__ void build_tables_kernel(int W, int H, int H_total, int y_off, int M, const double *abc, float *Xt,
                                    float *Yt, float *Xr, float *Yr, float2 *Xc, float2 *Yc, float *Y4t = nullptr,
                                    float *Y4r = nullptr, int ldy4 = 0, float2 *Yc2 = nullptr) {
  const long long total = (long long)M * (W + H);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(idx / (W + H)), i = (int)(idx % (W + H));
    const double am = abc[3 * m], bm = abc[3 * m + 1], cm = abc[3 * m + 2];
    double t;
    if (i < W) {
      const double q = (double)(i - W / 2);
      t = fma(cm * q, q, am * q);
    } else {
      const double q = (double)((i - W) + y_off - H_total / 2);
      t = fma(cm * q, q, bm * q);
    }
    t -= rint(t);  // [-1/2, 1/2] turns
    // turns (accurate mode); radians scaled by 1 + kFastEta (fast mode, see cis)
    const float tf = (float)t, rf = (float)(t * (6.283185307179586476925286766559 * (1.0 + (double)kFastEta)));
    double sn = 0.0, cs = 1.0;
    if (Xc) sincospi(2.0 * t, &sn, &cs);
    if (i < W) {
      Xt[(size_t)m * W + i] = tf;
      Xr[(size_t)m * W + i] = rf;
      if (Xc) Xc[(size_t)m * W + i] = make_float2((float)cs, (float)sn);
    } else {
      Yt[(size_t)m * H + (i - W)] = tf;
      Yr[(size_t)m * H + (i - W)] = rf;
      if (Y4t)
        for (int sh = 0; sh < 4; sh++) {
          Y4t[((size_t)sh * M + m) * ldy4 + (i - W) + sh] = tf;
          Y4r[((size_t)sh * M + m) * ldy4 + (i - W) + sh] = rf;
        }
      if (Yc) Yc[(size_t)m * H + (i - W)] = make_float2((float)cs, (float)sn);
      if (Yc2)
        for (int sh = 0; sh < 2; sh++) Yc2[((size_t)sh * M + m) * ldy4 + (i - W) + sh] = make_float2((float)cs, (float)sn);
    }
  }
}

// Fixed-point field sums -> float32 complex fields V_m (for callers of hot_field).
static __global__ void sums_to_fields_kernel(int M, const long long *Vsum, double inv, float2 *V) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < M) V[m] = make_float2((float)((double)Vsum[m] * inv), (float)((double)Vsum[M + m] * inv));
}

// Sec. 5 encoding of the phases: uint8 g = rint(phi 256 / 2pi) mod 256 (FP32 decision).
static __global__ void quantize_kernel(const float *phi, unsigned char *g, long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const float q = rintf(phi[j] * (256.0f / kTwoPi));
    g[j] = (unsigned char)(((int)q) & 255);
  }
}

}  // namespace hot
