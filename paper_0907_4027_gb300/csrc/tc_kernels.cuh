// tc_kernels.cuh -- the separable GSW iteration on the tensor cores (tcgen05, sm_103a).
//
// Eq. 2 is separable: e^{i Delta_j^m} = X_m(ix) Y_m(iy) with X_m(ix) = e^{i 2pi [a_m ix' + c_m ix'^2]}
// and Y_m(iy) = e^{i 2pi [b_m iy' + c_m iy'^2]}.  Both steps of a GSW iteration are then complex
// matrix products over the pixel grid:
//   back-projection (Sec. 4)  S[iy][ix] = sum_m (c_m Y_m(iy)) X_m(ix)        = P . X     (H x M by M x W)
//   forward field   (Eq. 1)   T[iy][m]  = sum_ix u[iy][ix] conj(X_m(ix))     = U . X^H   (H x W by W x M)
//                             N V_m     = sum_iy conj(Y_m(iy)) T[iy][m]
// with u = e^{i phi}.  Each complex product is one real GEMM on the 2x2 real embedding of the
// complex numbers: operands are stored complex-interleaved (real, imaginary) along K, and the
// constant right-hand operand holds the blocks [[xr, -xi], [xi, xr]] (back) or [[xr, xi], [-xi, xr]]
// (forward, the conjugate).  The GEMMs run on tcgen05.mma with FP32 accumulators in tensor
// memory.  A 16-bit or TF32 tensor-core operand keeps 11 significant bits, so every operand is
// split x = hi + lo and a product takes three MMAs, a_hi b_hi + a_hi b_lo + a_lo b_hi (the omitted
// a_lo b_lo is ~2^-22 relative): the products keep about FP32 accuracy.  The GSW iteration uses
// two FP16 parts (kind::f16: twice the TF32 rate, half the bytes; its operands are unit phasors and
// coefficients scaled to <= 1, where FP16 keeps its 11 bits); the GEMM also runs two TF32 parts
// (kind::tf32, the FP32 exponent range).
//
// A CTA computes one 128 x BN tile of a GEMM over a range of K, warp-specialised: one thread of
// warp 0 issues TMA loads of K slices (one 128-byte row per matrix row, 128-byte swizzle) of A_hi,
// A_lo, B_hi, B_lo into a ring of shared-memory stages; one thread of warp 1 issues the 12 MMAs of
// a slice into one of 2-4 tensor-memory accumulators and returns the stage to the loader with
// tcgen05.commit; the drain warps (TMEM lane quadrant = warp % 4, i.e. 32 rows each, and a group
// of <= 128 columns) add every slice's accumulator into FP32 registers while the MMAs of the next
// slices run in the other accumulators.  The tensor core's own accumulation into TMEM is not
// round-to-nearest (measured: a magnitude bias growing with the MMAs accumulated, ~1e-4 relative on
// small |V_m| after 190), so each accumulator holds the 12 MMAs of one slice only and the K sum
// runs in the registers (round-to-nearest, fixed order).  Then the epilogue:
//   back:    phi = arg S (atan2f), u = e^{i phi}, written as phases and as the split U operand;
//   forward: the tile's rows weighted by conj(Y_m(iy)) and summed, added into the 64-bit
//            fixed-point field accumulators (integer atomics: exact and order-independent, so
//            the K range may be split over CTAs);
//   plain:   C = A B^T (the GEMM alone, for tests).
// Every wait on an mbarrier is bounded by %globaltimer; when one runs out the CTA sets the error
// flag, stops issuing, waits (bounded) for the copies it has in flight, frees its tensor memory
// and returns.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tc {

constexpr int kBM = 128;         // rows of a tile: the 128 lanes of tensor memory
constexpr int kSliceBytes = 128; // one K slice per stage: one 128-byte swizzle row of every operand row
constexpr int kMmaKBytes = 32;   // K of one MMA: 8 TF32 or 16 FP16 elements

// Operand types.  TF32: FP32 storage, kind::tf32 (the MMA reads the top 19 bits).  FP16: halves,
// kind::f16 at twice the TF32 rate; its 11-bit significand equals TF32's, so the split keeps the
// same precision for operands of magnitude ~1 (the GSW operands are unit phasors and normalised
// coefficients), while subnormals limit it below ~2^-2 (the low part) and ~2^-14 (the high part).
constexpr int kOpTF32 = 0, kOpF16 = 1;
template <int OP>
struct Op;
template <>
struct Op<kOpTF32> {
  using T = float;
  static constexpr int kBytes = 4;
  static constexpr uint32_t kFmt = 2;  // instruction-descriptor operand format TF32
};
template <>
struct Op<kOpF16> {
  using T = __half;
  static constexpr int kBytes = 2;
  static constexpr uint32_t kFmt = 0;  // F16
};
template <int OP>
__host__ __device__ constexpr int slice_k() {  // K elements per slice: 32 (TF32) or 64 (FP16)
  return kSliceBytes / Op<OP>::kBytes;
}

constexpr int kEpiPlain = 0, kEpiBack = 1, kEpiFwd = 2;

// Tile width BN (32, 64, 128 or 256 columns): shared-memory stages as fit in 192 KB; the accumulator
// is drained by 4 warps per group of at most 128 columns (a thread keeps its row's columns of
// the group in registers), so BN = 256 has two column groups and 8 drain warps.
template <int BN>
struct Cfg {
  static_assert(BN == 32 || BN == 64 || BN == 128 || BN == 256, "tile width");
  static constexpr int kStages = BN == 256 ? 2 : BN == 128 ? 3 : 4;
  static constexpr int kABytes = kBM * kSliceBytes;  // 16 KB
  static constexpr int kBBytes = BN * kSliceBytes;
  static constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;
  static constexpr int kSmem = kStages * kStageBytes + 1024;  // + slack to align the ring to 1 KB
  static constexpr int kGroups = BN == 256 ? 2 : 1;           // column groups of the drain
  static constexpr int kCols = BN / kGroups;                  // columns per drain warp
  static constexpr int kEpiWarps = 4 * kGroups;               // one per TMEM lane quadrant and group
  static constexpr int kThreads = 32 * (2 + kEpiWarps);       // warp 0: TMA, warp 1: MMA, then drain
  static constexpr int kBufs = BN == 256 ? 2 : 4;             // accumulators in the 512 TMEM columns
  static constexpr int kTmemCols = kBufs * BN;                // a power of two >= 32
};
struct BackStage;

// The four operand maps of one GEMM (2-D, box of one 128-byte K slice x rows, 128-byte swizzle).
struct Maps {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
};

struct GemmArgs {
  int rows, cols;        // GEMM M and N: outputs outside are not written
  int k_chunks;          // K slices (K / slice_k)
  int chunks_per_split;  // K slices per CTA: CTA z takes slices z*cps .. min(k_chunks, (z+1)*cps)-1
  long long limit_ns;    // bound of every wait
  int *err;              // set to 1 when a wait runs out
  // plain
  float *C;              // [rows][cols]
  // back: S -> phi, U
  int W, H, Kf;          // pixels; row stride of U (elements)
  float *phi;            // [H][W]
  void *u_hi, *u_lo;     // [..][Kf] operand elements: (cos phi, sin phi) interleaved, split
  // forward: T -> fixed-point field sums
  int M;
  const float2 *Yc;              // [M][H] Y_m(iy)
  unsigned long long *acc_out;   // [2][M] Re, Im (zero before the first split adds)
  float fx_scale;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the completion of the phase of parity `parity`; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = timer_ns();
  for (;;) {
    for (int i = 0; i < 32; i++)
      if (mbar_try_wait(bar, parity)) return true;
    if ((long long)(timer_ns() - t0) > limit_ns) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile written by TMA with 128-byte
// swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), start address
// in 16-byte units; bits 46-47 = 1 (tcgen05 descriptor), bits 61-63 = 2 (128-byte swizzle).
// The leading byte offset is unused for a swizzled K-major tile whose K fits in one row.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::tf32 / kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// format at bits 7-9 and 10-12 (TF32 = 2, F16 = 0), both K-major (bits 15, 16 = 0), N >> 3 at
// bit 17, M >> 4 at bit 24.
template <int OP>
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
  return (1u << 4) | (Op<OP>::kFmt << 7) | (Op<OP>::kFmt << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

template <int OP>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  if (OP == kOpF16)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The barrier receives one arrival when every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes (thread t: lane 32w + t); the wait
// sits in the same statement, so the registers are complete when the statement ends.
__device__ __forceinline__ void tmem_load32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void grid_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void grid_release() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// x ~ hi + lo, both exactly representable in the operand type (returned as floats).  TF32: hi is
// x with the 13 low mantissa bits cleared, lo the exact FP32 rest (the MMA reads its TF32 part).
// FP16: hi = x rounded to half, lo = the rest rounded to half.
template <int OP>
__device__ __forceinline__ float2 split2(float x) {
  if (OP == kOpF16) {
    const float hi = __half2float(__float2half_rn(x));
    return make_float2(hi, __half2float(__float2half_rn(x - hi)));
  }
  const float hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  return make_float2(hi, x - hi);
}

// Element i of an operand array (a value split2 produced, so the conversion is exact).
template <int OP>
__device__ __forceinline__ void store1(void *base, size_t i, float v) {
  if (OP == kOpF16)
    static_cast<__half *>(base)[i] = __float2half_rn(v);
  else
    static_cast<float *>(base)[i] = v;
}
// Elements i, i + 1 (i even).
template <int OP>
__device__ __forceinline__ void store2(void *base, size_t i, float a, float b) {
  if (OP == kOpF16)
    *reinterpret_cast<__half2 *>(static_cast<__half *>(base) + i) = __floats2half2_rn(a, b);
  else
    *reinterpret_cast<float2 *>(static_cast<float *>(base) + i) = make_float2(a, b);
}

// u = e^{i phi} of a phase in any range: reduced to [-pi, pi] (Cody-Waite with 2 pi split in
// two floats; a no-op for the back-projection's own phases in (-pi, pi]), then the SFU's
// sin/cos approximations (|error| ~ 4e-7 on that interval).  The forward operand of the phases
// a call starts from and of the phases an iteration writes come from this one function, so a
// resumed run repeats the bits of an uninterrupted one.
__device__ __forceinline__ void unit_phasor(float ph, float &sn, float &cs) {
  const float k = rintf(ph * 0.15915494309189535f);
  const float x = fmaf(-k, -1.74845553e-07f, fmaf(-k, 6.28318548e+00f, ph));
  __sincosf(x, &sn, &cs);
}

// Stores a complex value split into the hi and lo operand arrays at element i (even).
template <int OP>
__device__ __forceinline__ void store_split(void *hi, void *lo, size_t i, float re, float im) {
  const float2 r = split2<OP>(re), m = split2<OP>(im);
  store2<OP>(hi, i, r.x, m.x);
  store2<OP>(lo, i, r.y, m.y);
}

// 32 accumulator columns n0 .. n0+31 of one row of the plain GEMM: C.
__device__ __forceinline__ void epilogue_plain(const GemmArgs &a, const float *v, int row, int n0) {
  if (row < a.rows)
#pragma unroll
    for (int c = 0; c < 32; c++)
      if (n0 + c < a.cols) a.C[(size_t)row * a.cols + n0 + c] = v[c];
}

// Back-projection: 32 accumulator columns n0 .. n0+31, columns 2 p, 2 p + 1 = Re S, Im S of pixel
// ix = n0/2 + p of this thread's row -> phi = arg S (Sec. 4; atan2(0, 0) = 0) and u = e^{i phi}.
// A thread holds one row, so the 16 pixels are first written to the warp's staging area in
// shared memory (rows padded against bank conflicts) and then stored row segment by row segment:
// each store instruction of the warp writes whole 32-byte sectors of one or two rows instead
// of one word in each of 32 rows.
struct BackStage {
  float ph[32][17];  // phases of 16 pixels of 32 rows
  float uh[32][33];  // (cos, sin) interleaved, high parts
  float ul[32][33];  // and low parts
};
template <int OP>
__device__ __forceinline__ void epilogue_back(const GemmArgs &a, const float *v, int row0, int n0, BackStage &st) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int p = 0; p < 16; p++) {
    const float ph = atan2f(v[2 * p + 1], v[2 * p]);
    float sn, cs;
    unit_phasor(ph, sn, cs);
    const float2 c2 = split2<OP>(cs), s2 = split2<OP>(sn);
    st.ph[lane][p] = ph;
    st.uh[lane][2 * p] = c2.x;
    st.uh[lane][2 * p + 1] = s2.x;
    st.ul[lane][2 * p] = c2.y;
    st.ul[lane][2 * p + 1] = s2.y;
  }
  __syncwarp();
  const int x0 = n0 >> 1;
#pragma unroll 4
  for (int i = 0; i < 16; i++) {  // phases: two rows of 16 pixels per instruction
    const int r = 2 * i + (lane >> 4), p = lane & 15, iy = row0 + r, ix = x0 + p;
    if (iy < a.H && ix < a.W) a.phi[(size_t)iy * a.W + ix] = st.ph[r][p];
  }
#pragma unroll 4
  for (int r = 0; r < 32; r++) {  // operand: one row of 16 pixels (128 bytes) per instruction
    const int iy = row0 + r, ix = x0 + (lane >> 1);
    if (iy < a.H && ix < a.W) {
      const size_t o = (size_t)iy * a.Kf + 2 * x0 + lane;
      store1<OP>(a.u_hi, o, st.uh[r][lane]);
      store1<OP>(a.u_lo, o, st.ul[r][lane]);
    }
  }
  __syncwarp();
}

// Forward: the warp's COLS columns c0 .. c0+COLS-1 of the tile (2 p, 2 p + 1 = Re, Im of T[row][m],
// m = (n0 + c0)/2 + p).  The terms T conj(Y_m(row)) are summed over the tile's 128 rows (in each
// warp a transposed shuffle reduction after which lane L holds columns COLS/32 L ..; then the four
// lane quadrants in order) and added into the fixed-point sums, one atomic per trap and component.
// q: the warp's TMEM lane quadrant, g its column group; ok: its accumulator is complete; failed:
// the CTA's flag, read after the drain warps' barrier (an incomplete tile adds nothing).
template <int BN>
__device__ __forceinline__ void epilogue_fwd(const GemmArgs &a, float *z, int row, int n0, float *red, int q, int g,
                                             bool ok, const int *failed) {
  constexpr int COLS = Cfg<BN>::kCols, PER = COLS / 32;
  const int mt0 = (n0 + g * COLS) >> 1;
#pragma unroll
  for (int p = 0; p < COLS / 2; p++) {
    const int m = mt0 + p;
    const float tr = z[2 * p], ti = z[2 * p + 1];
    float zr = 0.f, zi = 0.f;
    if (ok && row < a.H && m < a.M) {
      const float2 y = __ldg(a.Yc + (size_t)m * a.H + row);
      zr = fmaf(tr, y.x, ti * y.y);
      zi = fmaf(ti, y.x, -tr * y.y);
    }
    z[2 * p] = zr;
    z[2 * p + 1] = zi;
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16, n = COLS; o >= 1; o >>= 1, n >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; i++) {
      const float send = upper ? z[i] : z[i + n / 2];
      const float keep = upper ? z[i + n / 2] : z[i];
      z[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (int i = 0; i < PER; i++) red[(g * 4 + q) * COLS + PER * lane + i] = z[i];
  asm volatile("bar.sync 1, %0;" ::"n"(32 * Cfg<BN>::kEpiWarps) : "memory");  // the drain warps only
  const int t = threadIdx.x - 64;  // index among the drain threads
  if (t < BN && !*(const volatile int *)failed) {
    const int gg = t / COLS, j = t % COLS;
    const int m = (n0 + t) >> 1;
    if (m < a.M) {
      const float *r = red + gg * 4 * COLS + j;
      const float s = ((r[0] + r[COLS]) + r[2 * COLS]) + r[3 * COLS];
      // |s| <= N, so s * 2^fx_shift rounds to an integer below 2^61
      atomicAdd(a.acc_out + (size_t)(t & 1) * a.M + m, (unsigned long long)__float2ll_rn(s * a.fx_scale));
    }
  }
}

// One 128 x BN output tile over a K range: TMA loader (warp 0, one lane), MMA issuer (warp 1,
// one lane), accumulator drain and epilogue (the other warps).  grid = (N tiles, M tiles, K splits).
template <int BN, int EPI, int OP>
__global__ void __launch_bounds__(Cfg<BN>::kThreads, 1) tc_gemm_kernel(const __grid_constant__ Maps maps,
                                                                       const __grid_constant__ GemmArgs a) {
  using C = Cfg<BN>;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[C::kStages], empty[C::kStages], tfull[C::kBufs], tempty[C::kBufs];
  __shared__ uint32_t tmem_slot;
  __shared__ int issued, consumed, failed;
  __shared__ float red[EPI == kEpiFwd ? 4 * BN : 1];
  // the ring starts on a 1 KB boundary of the shared window (the 128-byte swizzle pattern repeats
  // every 8 rows of 128 bytes and the descriptors assume aligned tiles)
  unsigned char *ring = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * kBM;
  const int kc0 = blockIdx.z * a.chunks_per_split;
  const int nk = min(a.k_chunks - kc0, a.chunks_per_split);  // >= 1 (the host sizes the splits)
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < C::kBufs; b++) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], C::kEpiWarps);
    }
    issued = consumed = failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.a_hi)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.b_hi)) : "memory");
  }
  if (warp == 0) {  // the whole warp allocates kBufs FP32 accumulators of BN columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(C::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  grid_wait();  // the A operand is the previous kernel's output
  grid_release();

  if (warp == 0) {
    if (lane == 0) {
      for (int i = 0; i < nk; i++) {
        const int s = i % C::kStages;
        const uint32_t ph = (uint32_t)(i / C::kStages) & 1u;
        if (i >= C::kStages && !mbar_wait(&empty[s], ph ^ 1u, a.limit_ns)) {
          failed = 1;
          break;
        }
        if (*(volatile int *)&failed) break;
        unsigned char *st = ring + s * C::kStageBytes;
        mbar_expect_tx(&full[s], C::kStageBytes);
        const int kx = (kc0 + i) * slice_k<OP>();
        tma_load_2d(st, &maps.a_hi, kx, m0, &full[s]);
        tma_load_2d(st + C::kABytes, &maps.a_lo, kx, m0, &full[s]);
        tma_load_2d(st + 2 * C::kABytes, &maps.b_hi, kx, n0, &full[s]);
        tma_load_2d(st + 2 * C::kABytes + C::kBBytes, &maps.b_lo, kx, n0, &full[s]);
        *(volatile int *)&issued = i + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = instr_desc<OP>(kBM, BN);
      for (int i = 0; i < nk; i++) {
        const int b = i % C::kBufs;
        // accumulator b is free once the drain warps have emptied its previous slice
        if (i >= C::kBufs && !mbar_wait(&tempty[b], (uint32_t)(i / C::kBufs - 1) & 1u, a.limit_ns)) {
          failed = 1;
          break;
        }
        const int s = i % C::kStages;
        const uint32_t ph = (uint32_t)(i / C::kStages) & 1u;
        if (*(volatile int *)&failed || !mbar_wait(&full[s], ph, a.limit_ns)) {
          failed = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(ring + s * C::kStageBytes);
        const uint32_t d = tmem + (uint32_t)(b * BN);
#pragma unroll
        for (int kk = 0; kk < kSliceBytes / kMmaKBytes; kk++) {
          const uint32_t off = kk * kMmaKBytes;  // 32 bytes per MMA step along K
          const uint64_t ahi = smem_desc(sa + off), alo = smem_desc(sa + C::kABytes + off);
          const uint64_t bhi = smem_desc(sa + 2 * C::kABytes + off);
          const uint64_t blo = smem_desc(sa + 2 * C::kABytes + C::kBBytes + off);
          mma<OP>(d, ahi, bhi, idesc, kk != 0);
          mma<OP>(d, ahi, blo, idesc, 1u);
          mma<OP>(d, alo, bhi, idesc, 1u);
        }
        mma_commit(&empty[s]);  // the stage returns to the loader when these MMAs have read it
        mma_commit(&tfull[b]);  // and the accumulator goes to the epilogue warps
        *(volatile int *)&consumed = i + 1;
      }
    }
    __syncwarp();
  } else {
    // drain: slice i's partial product (accumulator i % kBufs) added into registers in slice order
    constexpr int COLS = C::kCols;
    const int q = warp & 3;          // TMEM lane quadrant of this warp: rows 32q .. 32q+31
    const int g = (warp - 2) >> 2;   // its column group: columns g COLS .. (g+1) COLS - 1
    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * COLS);
    float acc[COLS];
#pragma unroll
    for (int c = 0; c < COLS; c++) acc[c] = 0.f;
    bool ok = true;
    for (int i = 0; i < nk; i++) {
      const int b = i % C::kBufs;
      ok = mbar_wait(&tfull[b], (uint32_t)(i / C::kBufs) & 1u, a.limit_ns);
      ok = __all_sync(0xffffffffu, ok) && !*(volatile int *)&failed;
      if (!ok) break;
      tc_fence_after();
#pragma unroll
      for (int c = 0; c < COLS; c += 32) {
        float v[32];
        tmem_load32(tq + (uint32_t)(b * BN + c), v);
#pragma unroll
        for (int j = 0; j < 32; j++) acc[c + j] += v[j];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
    if (!ok && lane == 0) {
      failed = 1;
      atomicExch(a.err, 1);
    }
    const int row = m0 + q * 32 + lane;
    if (EPI == kEpiFwd) {
      epilogue_fwd<BN>(a, acc, row, n0, red, q, g, ok, &failed);
    } else if (EPI == kEpiBack && ok) {
      static_assert(sizeof(BackStage) * C::kEpiWarps <= C::kStages * C::kStageBytes, "staging fits the ring");
      // the ring is free: every MMA that read it has completed (the last slice was drained)
      BackStage &st = reinterpret_cast<BackStage *>(ring)[warp - 2];
#pragma unroll
      for (int c = 0; c < COLS; c += 32) epilogue_back<OP>(a, acc + c, m0 + q * 32, n0 + g * COLS + c, st);
    } else if (ok) {
#pragma unroll
      for (int c = 0; c < COLS; c += 32) epilogue_plain(a, acc + c, row, n0 + g * COLS + c);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && failed) {
    atomicExch(a.err, 1);
    // copies still in flight: wait (bounded) until they have landed before the CTA exits
    for (int i = consumed; i < issued; i++) mbar_wait(&full[i % C::kStages], (uint32_t)(i / C::kStages) & 1u, a.limit_ns);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kTmemCols) : "memory");
  }
}

// ---------------------------------------------------------------------------------------------
// Operand preparation

// Constant right-hand operands from the complex column tables Xc[m][ix] (once per trap set):
//   back    Bb[n][k], n = 2 ix + r, k = 2 m + s: [[xr, -xi], [xi, xr]][r][s]    (2W x Kb)
//   forward Bf[n][k], n = 2 m + r,  k = 2 ix + s: [[xr, xi], [-xi, xr]][r][s]   (2M x Kf)
// and the row table transposed, YT[iy][m] = Y_m(iy) (m < Kb/2, zero beyond M).  Padding rows and
// columns are zero.  Rows of Bb and Bf are padded to the tile width, Kb and Kf to a K slice.
struct TableArgs {
  int W, H, M, Kb, Kf, rows_b, rows_f;
  const float2 *Xc, *Yc;
  void *bb_hi, *bb_lo, *bf_hi, *bf_lo;  // operand elements
  float2 *YT;
};

template <int OP>
__global__ void tc_tables_kernel(TableArgs a) {
  const long long nb = (long long)a.rows_b * a.Kb, nf = (long long)a.rows_f * a.Kf;
  const long long ny = (long long)a.H * (a.Kb / 2);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb + nf + ny; i += stride) {
    if (i < nb) {
      const int n = (int)(i / a.Kb), k = (int)(i % a.Kb);
      const int ix = n >> 1, r = n & 1, m = k >> 1, s = k & 1;
      float val = 0.f;
      if (ix < a.W && m < a.M) {
        const float2 x = a.Xc[(size_t)m * a.W + ix];
        val = (r == s) ? x.x : (r == 0 ? -x.y : x.y);
      }
      const float2 h = split2<OP>(val);
      store1<OP>(a.bb_hi, i, h.x);
      store1<OP>(a.bb_lo, i, h.y);
    } else if (i < nb + nf) {
      const long long j = i - nb;
      const int n = (int)(j / a.Kf), k = (int)(j % a.Kf);
      const int m = n >> 1, r = n & 1, ix = k >> 1, s = k & 1;
      float val = 0.f;
      if (ix < a.W && m < a.M) {
        const float2 x = a.Xc[(size_t)m * a.W + ix];
        val = (r == s) ? x.x : (r == 0 ? x.y : -x.y);
      }
      const float2 h = split2<OP>(val);
      store1<OP>(a.bf_hi, j, h.x);
      store1<OP>(a.bf_lo, j, h.y);
    } else {
      const long long j = i - nb - nf;
      const int iy = (int)(j / (a.Kb / 2)), m = (int)(j % (a.Kb / 2));
      a.YT[j] = m < a.M ? a.Yc[(size_t)m * a.H + iy] : make_float2(0.f, 0.f);
    }
  }
}

// The forward operand of given phases: u = e^{i phi} (unit_phasor), split; and one accumulator
// buffer cleared for the launch after next.
template <int OP>
__global__ void tc_phase_kernel(int W, int H, int Kf, const float *phi, void *u_hi, void *u_lo,
                                unsigned long long *acc_clear, int n_clear) {
  grid_wait();
  const long long N = (long long)W * H, stride = (long long)gridDim.x * blockDim.x;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < N; j += stride) {
    const int iy = (int)(j / W), ix = (int)(j % W);
    float sn, cs;
    unit_phasor(phi[j], sn, cs);
    store_split<OP>(u_hi, u_lo, (size_t)iy * Kf + 2 * ix, cs, sn);
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_clear; i += stride) acc_clear[i] = 0ull;
  grid_release();
}

struct PrepArgs {
  int H, M, Kb;
  const unsigned long long *acc_in;  // [2][M] sums of the previous forward
  unsigned long long *acc_clear;     // [2][M] cleared here
  const float *w_in;
  float *w_out;                      // written by block 0
  const float2 *YT;                  // [H][Kb/2]
  void *p_hi, *p_lo;                 // [..][Kb] operand elements
  float inv_fx_n;
  float *trace;                      // NULL, or e, u of the fields read (block 0)
};

struct ffp {
  float hi, lo;
};
__device__ __forceinline__ ffp ffp_add(ffp a, ffp b) {  // TwoSum (Knuth) + renormalisation
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b.hi - bb);
  const float e = err + (a.lo + b.lo);
  const float hi = s + e;
  return {hi, e - (hi - s)};
}

constexpr int kPrepThreads = 256;
constexpr int kPrepPrefetch = 16;  // row-table elements a thread of tc_prep_kernel fetches before the wait

// Sec. 3 weight update and the back-projection operand of one iteration: every block reads the
// field sums, forms V_m, <|V|> (float-float sum in one fixed order, so every block obtains the
// same bits) and the coefficients c_m = w_m' V_m/|V_m| with w_m' = w_m <|V|>/|V_m| (|V_m| < 1e-30:
// c_m = w_m, w kept) in shared memory, then writes its share of P[iy][2m..2m+1] = c_m Y_m(iy),
// split.  Block 0 writes the new weights (and the trace); the blocks clear the next buffer.
// The row table is constant during hot_gsw: a thread's first kPrepPrefetch elements of it are
// fetched before the wait for the previous kernel (they come from HBM: the GEMMs' operands have
// pushed the table out of L2).
template <int OP>
__global__ void __launch_bounds__(kPrepThreads) tc_prep_kernel(PrepArgs a) {
  extern __shared__ float2 cs[];  // [M]
  __shared__ ffp part[2][kPrepThreads / 32];
  __shared__ float ext[2][kPrepThreads / 32];
  __shared__ float cmx[kPrepThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // this block's rows of P: an even share of the H rows, all Kb/2 (padded) traps of each
  const int half = a.Kb / 2;
  const int r0 = (int)((long long)a.H * blockIdx.x / gridDim.x);
  const int r1 = (int)((long long)a.H * (blockIdx.x + 1) / gridDim.x);
  const int n = (r1 - r0) * half;
  float2 ypre[kPrepPrefetch];
#pragma unroll
  for (int j = 0; j < kPrepPrefetch; j++) {
    const int i = t + j * kPrepThreads;
    ypre[j] = i < n ? __ldg(a.YT + (size_t)r0 * half + i) : make_float2(0.f, 0.f);
  }
  grid_wait();
  ffp s = {0.f, 0.f}, si = {0.f, 0.f};
  float mx = -1.f, mn = 3.0e38f;
  for (int m = t; m < a.M; m += kPrepThreads) {
    const float vr = (float)(long long)__ldcg(a.acc_in + m) * a.inv_fx_n;
    const float vi = (float)(long long)__ldcg(a.acc_in + a.M + m) * a.inv_fx_n;
    cs[m] = make_float2(vr, vi);
    const float I = vr * vr + vi * vi;
    s = ffp_add(s, {sqrtf(I), 0.f});
    si = ffp_add(si, {I, 0.f});
    mx = fmaxf(mx, I);
    mn = fminf(mn, I);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    s = ffp_add(s, {__shfl_down_sync(0xffffffffu, s.hi, o), __shfl_down_sync(0xffffffffu, s.lo, o)});
    si = ffp_add(si, {__shfl_down_sync(0xffffffffu, si.hi, o), __shfl_down_sync(0xffffffffu, si.lo, o)});
    mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
  }
  if (lane == 0) {
    part[0][warp] = s;
    part[1][warp] = si;
    ext[0][warp] = mx;
    ext[1][warp] = mn;
  }
  __syncthreads();
  ffp q = part[0][0];
  for (int i = 1; i < kPrepThreads / 32; i++) q = ffp_add(q, part[0][i]);
  const float mean = (q.hi + q.lo) / (float)a.M;  // <|V|> (Sec. 3)
  if (a.trace && blockIdx.x == 0 && t == 0) {  // e, u (Eq. 4) of the fields read
    ffp e = part[1][0];
    float hi = ext[0][0], lo = ext[1][0];
    for (int i = 1; i < kPrepThreads / 32; i++) {
      e = ffp_add(e, part[1][i]);
      hi = fmaxf(hi, ext[0][i]);
      lo = fminf(lo, ext[1][i]);
    }
    a.trace[0] = e.hi + e.lo;
    a.trace[1] = (hi + lo > 0.f) ? 1.f - (hi - lo) / (hi + lo) : 0.f;
  }
  float cmax = 0.f;  // largest |c_m| (= w_m'): the coefficients are scaled by its inverse below
  for (int m = t; m < a.M; m += kPrepThreads) {
    const float2 v = cs[m];
    const float w = __ldcg(a.w_in + m);
    const float am = sqrtf(v.x * v.x + v.y * v.y);
    float2 c;
    float wn = w;
    if (am < 1e-30f) {
      c = make_float2(w, 0.f);
    } else {
      wn = w * mean / am;
      c = make_float2(wn * (v.x / am), wn * (v.y / am));
    }
    if (blockIdx.x == 0) a.w_out[m] = wn;
    cs[m] = c;
    cmax = fmaxf(cmax, wn);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
  if (lane == 0) cmx[warp] = cmax;
  const long long stride = (long long)gridDim.x * kPrepThreads;
  for (long long i = blockIdx.x * (long long)kPrepThreads + t; i < 2LL * a.M; i += stride) a.acc_clear[i] = 0ull;
  __syncthreads();
  // A factor common to all coefficients leaves arg S unchanged (Sec. 4; the weights' scale is
  // free): P is formed from c_m / max |c| so that its magnitudes stay near 1 whatever the
  // weights' scale (the FP16 operands lose precision below ~0.25).
  float top = cmx[0];
  for (int i = 1; i < kPrepThreads / 32; i++) top = fmaxf(top, cmx[i]);
  const float scale = top > 0.f ? 1.f / top : 1.f;
  // element i of the block's rows is P[r0 + i / half][m = i % half], at i of the row-major table
  auto put = [&](int i, float2 y) {
    const int m = i % half;
    const float2 c = m < a.M ? make_float2(cs[m].x * scale, cs[m].y * scale) : make_float2(0.f, 0.f);
    store_split<OP>(a.p_hi, a.p_lo, 2 * ((size_t)r0 * half + i), c.x * y.x - c.y * y.y, c.x * y.y + c.y * y.x);
  };
#pragma unroll
  for (int j = 0; j < kPrepPrefetch; j++)
    if (t + j * kPrepThreads < n) put(t + j * kPrepThreads, ypre[j]);
  for (int i = t + kPrepPrefetch * kPrepThreads; i < n; i += kPrepThreads) put(i, __ldg(a.YT + (size_t)r0 * half + i));
  grid_release();
}

// Operands of the plain GEMM entry point: src [rows][K] -> hi, lo [rows_pad][K_pad], zero padded.
template <int OP>
__global__ void tc_split_kernel(const float *src, int rows, int K, int K_pad, long long total, void *hi, void *lo) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / K_pad), k = (int)(i % K_pad);
    const float x = (r < rows && k < K) ? src[(size_t)r * K + k] : 0.f;
    const float2 h = split2<OP>(x);
    store1<OP>(hi, i, h.x);
    store1<OP>(lo, i, h.y);
  }
}

}  // namespace tc
