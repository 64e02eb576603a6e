// tc.cu -- host side of the separable GSW iteration on the tensor cores (see tc_kernels.cuh).
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "tc.h"
#include "tc_kernels.cuh"

namespace hot_tc {

// Operand type of the GSW iteration's GEMMs: FP16 halves (kind::f16, twice the TF32 rate; the
// operands are unit phasors and coefficients normalised to max |c_m| = 1).
constexpr int kPlanOp = tc::kOpF16;
constexpr int kSliceK = tc::slice_k<kPlanOp>();
constexpr size_t kElem = tc::Op<kPlanOp>::kBytes;

struct Plan {
  int W = 0, H = 0, M = 0;
  int Kb = 0, Kf = 0;               // K of the back GEMM (2M) and forward GEMM (2W), padded to a K slice
  int rows_h = 0;                   // H padded to the tile height (rows of P and U)
  int bn_back = 64, bn_fwd = 64;    // tile widths of the back and forward GEMMs
  int rows_b = 0, rows_f = 0;       // rows of Bb (2W) and Bf (2M), padded to the tile width
  int fwd_splits = 1, fwd_cps = 1;  // K splits of the forward GEMM, K slices per split
  int sms = 0;
  void *bb_hi = nullptr, *bb_lo = nullptr, *bf_hi = nullptr, *bf_lo = nullptr;  // operand elements
  void *p_hi = nullptr, *p_lo = nullptr, *u_hi = nullptr, *u_lo = nullptr;
  float2 *YT = nullptr;
  const float2 *Xc = nullptr, *Yc = nullptr;  // the context's complex tables [M][W], [M][H]
  tc::Maps back{}, fwd{};
};

namespace {

int round_up(int x, int m) { return (x + m - 1) / m * m; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// A row-major operand matrix [rows][inner] of OP elements (inner a multiple of one K slice, base
// 16-byte aligned) read in boxes of one 128-byte K slice x box_rows with 128-byte swizzle; rows
// is a multiple of box_rows, so no box leaves the matrix.
template <int OP>
cudaError_t encode(CUtensorMap *map, const void *base, int inner, int rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)inner * tc::Op<OP>::kBytes};
  const cuuint32_t box[2] = {(cuuint32_t)tc::slice_k<OP>(), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = OP == tc::kOpF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const CUresult r = fn(map, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename... KArgs, typename... Args>
cudaError_t launch(void (*kernel)(KArgs...), dim3 grid, int block, int smem, cudaStream_t st, bool pdl,
                   Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int BN, int EPI, int OP = kPlanOp>
cudaError_t set_smem() {
  return cudaFuncSetAttribute(tc::tc_gemm_kernel<BN, EPI, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              tc::Cfg<BN>::kSmem);
}

template <typename T>
cudaError_t alloc(T **p, size_t count) {
  return cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
}
cudaError_t alloc_bytes(void **p, size_t bytes) { return cudaMalloc(p, bytes); }

template <int BN, int EPI, int OP = kPlanOp>
cudaError_t launch_gemm(const tc::Maps &maps, const tc::GemmArgs &g, dim3 grid, cudaStream_t st, bool pdl) {
  return launch(tc::tc_gemm_kernel<BN, EPI, OP>, grid, tc::Cfg<BN>::kThreads, tc::Cfg<BN>::kSmem, st, pdl, maps, g);
}

template <int EPI>
cudaError_t launch_gemm_bn(int bn, const tc::Maps &maps, const tc::GemmArgs &g, dim3 grid, cudaStream_t st, bool pdl) {
  return bn == 256 ? launch_gemm<256, EPI>(maps, g, grid, st, pdl)
         : bn == 128 ? launch_gemm<128, EPI>(maps, g, grid, st, pdl)
         : bn == 64  ? launch_gemm<64, EPI>(maps, g, grid, st, pdl)
                     : launch_gemm<32, EPI>(maps, g, grid, st, pdl);
}

// Tile width of a GEMM with `rows` x `cols` outputs: the widest whose tiles still occupy most
// SMs and add little padding (wider tiles load fewer operand bytes per MMA; L2 bandwidth bounds
// the narrow ones).
// split_k: the K range may be split over CTAs (the forward GEMM) when it has >= 4 slices each.
int pick_width(int rows, int cols, int k_chunks, int sms, bool split_k) {
  for (int bn : {256, 128, 64}) {
    if (8 * round_up(cols, bn) > 9 * round_up(cols, 32)) continue;  // > 12.5% more padding than 32
    const long long tiles = (long long)((rows + tc::kBM - 1) / tc::kBM) * ((cols + bn - 1) / bn);
    const long long ctas = split_k ? tiles * std::max(1, std::min(k_chunks / 4, sms / (int)std::max(1LL, tiles)))
                                   : tiles;
    if (ctas * 5 >= 4LL * sms) return bn;
  }
  return 32;
}

}  // namespace

Shape shape_for(int W, int H, int M, int sms) {
  Shape sh;
  sh.Kb = round_up(2 * M, kSliceK);
  sh.Kf = round_up(2 * W, kSliceK);
  sh.rows_h = round_up(H, tc::kBM);
  sh.bn_back = pick_width(H, 2 * W, sh.Kb / kSliceK, sms, false);
  sh.bn_fwd = pick_width(H, 2 * M, sh.Kf / kSliceK, sms, true);
  sh.rows_b = round_up(2 * W, sh.bn_back);
  sh.rows_f = round_up(2 * M, sh.bn_fwd);
  // forward GEMM: the K range split over CTAs so that the tiles fill the SMs about once
  const int tiles_f = (sh.rows_h / tc::kBM) * (sh.rows_f / sh.bn_fwd);
  const int kcf = sh.Kf / kSliceK;
  const int splits = std::max(1, std::min(kcf, sms / std::max(tiles_f, 1)));
  sh.fwd_cps = (kcf + splits - 1) / splits;
  sh.fwd_splits = (kcf + sh.fwd_cps - 1) / sh.fwd_cps;  // every split has >= 1 slice
  return sh;
}

void plan_destroy(Plan *p) {
  if (!p) return;
  for (void *b : {p->bb_hi, p->bb_lo, p->bf_hi, p->bf_lo, p->p_hi, p->p_lo, p->u_hi, p->u_lo})
    if (b) cudaFree(b);
  if (p->YT) cudaFree(p->YT);
  delete p;
}

cudaError_t plan_refresh(Plan *p, cudaStream_t st) {
  tc::TableArgs t = {};
  t.W = p->W;
  t.H = p->H;
  t.M = p->M;
  t.Kb = p->Kb;
  t.Kf = p->Kf;
  t.rows_b = p->rows_b;
  t.rows_f = p->rows_f;
  t.Xc = p->Xc;
  t.Yc = p->Yc;
  t.bb_hi = p->bb_hi;
  t.bb_lo = p->bb_lo;
  t.bf_hi = p->bf_hi;
  t.bf_lo = p->bf_lo;
  t.YT = p->YT;
  const long long total = (long long)p->rows_b * p->Kb + (long long)p->rows_f * p->Kf + (long long)p->H * (p->Kb / 2);
  const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * p->sms);
  return launch(tc::tc_tables_kernel<kPlanOp>, dim3(blocks), 256, 0, st, false, t);
}

cudaError_t plan_create(Plan **out, int W, int H, int M, const float2 *Xc, const float2 *Yc, cudaStream_t st,
                        const char **what) {
  *out = nullptr;
  Plan *p = new Plan;
  p->W = W;
  p->H = H;
  p->M = M;
  p->Xc = Xc;
  p->Yc = Yc;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev);
  const Shape sh = shape_for(W, H, M, p->sms);
  p->Kb = sh.Kb;
  p->Kf = sh.Kf;
  p->rows_h = sh.rows_h;
  p->bn_back = sh.bn_back;
  p->bn_fwd = sh.bn_fwd;
  p->rows_b = sh.rows_b;
  p->rows_f = sh.rows_f;
  p->fwd_cps = sh.fwd_cps;
  p->fwd_splits = sh.fwd_splits;
  *what = "allocating the tensor-core operands";
  const size_t nb = (size_t)p->rows_b * p->Kb, nf = (size_t)p->rows_f * p->Kf;
  const size_t np = (size_t)p->rows_h * p->Kb, nu = (size_t)p->rows_h * p->Kf;
  if (e == cudaSuccess) e = alloc_bytes(&p->bb_hi, nb * kElem);
  if (e == cudaSuccess) e = alloc_bytes(&p->bb_lo, nb * kElem);
  if (e == cudaSuccess) e = alloc_bytes(&p->bf_hi, nf * kElem);
  if (e == cudaSuccess) e = alloc_bytes(&p->bf_lo, nf * kElem);
  if (e == cudaSuccess) e = alloc_bytes(&p->p_hi, np * kElem);
  if (e == cudaSuccess) e = alloc_bytes(&p->p_lo, np * kElem);
  if (e == cudaSuccess) e = alloc_bytes(&p->u_hi, nu * kElem);
  if (e == cudaSuccess) e = alloc_bytes(&p->u_lo, nu * kElem);
  if (e == cudaSuccess) e = alloc(&p->YT, (size_t)H * (p->Kb / 2));
  // padding rows and columns of P and U stay zero (the kernels write only the image)
  if (e == cudaSuccess) e = cudaMemsetAsync(p->p_hi, 0, np * kElem, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->p_lo, 0, np * kElem, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->u_hi, 0, nu * kElem, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->u_lo, 0, nu * kElem, st);
  if (e == cudaSuccess) {
    *what = "building the tensor-core operand tables";
    e = plan_refresh(p, st);
  }
  if (e == cudaSuccess) {
    *what = "encoding the tensor maps";
    e = encode<kPlanOp>(&p->back.a_hi, p->p_hi, p->Kb, p->rows_h, tc::kBM);
    if (e == cudaSuccess) e = encode<kPlanOp>(&p->back.a_lo, p->p_lo, p->Kb, p->rows_h, tc::kBM);
    if (e == cudaSuccess) e = encode<kPlanOp>(&p->back.b_hi, p->bb_hi, p->Kb, p->rows_b, p->bn_back);
    if (e == cudaSuccess) e = encode<kPlanOp>(&p->back.b_lo, p->bb_lo, p->Kb, p->rows_b, p->bn_back);
    if (e == cudaSuccess) e = encode<kPlanOp>(&p->fwd.a_hi, p->u_hi, p->Kf, p->rows_h, tc::kBM);
    if (e == cudaSuccess) e = encode<kPlanOp>(&p->fwd.a_lo, p->u_lo, p->Kf, p->rows_h, tc::kBM);
    if (e == cudaSuccess) e = encode<kPlanOp>(&p->fwd.b_hi, p->bf_hi, p->Kf, p->rows_f, p->bn_fwd);
    if (e == cudaSuccess) e = encode<kPlanOp>(&p->fwd.b_lo, p->bf_lo, p->Kf, p->rows_f, p->bn_fwd);
  }
  if (e == cudaSuccess) {
    *what = "setting the tensor-core kernels' shared memory";
    e = set_smem<32, tc::kEpiBack>();
    if (e == cudaSuccess) e = set_smem<64, tc::kEpiBack>();
    if (e == cudaSuccess) e = set_smem<128, tc::kEpiBack>();
    if (e == cudaSuccess) e = set_smem<256, tc::kEpiBack>();
    if (e == cudaSuccess) e = set_smem<32, tc::kEpiFwd>();
    if (e == cudaSuccess) e = set_smem<64, tc::kEpiFwd>();
    if (e == cudaSuccess) e = set_smem<128, tc::kEpiFwd>();
    if (e == cudaSuccess) e = set_smem<256, tc::kEpiFwd>();
  }
  if (e != cudaSuccess) {
    cudaStreamSynchronize(st);
    plan_destroy(p);
    return e;
  }
  *out = p;
  return cudaSuccess;
}

cudaError_t launch_forward(Plan *p, const Step &s, cudaStream_t st, bool pdl, bool chain, int *kernels) {
  *kernels = 0;
  const long long N = (long long)p->W * p->H;
  const int blocks = (int)std::min<long long>((N + 255) / 256, 8LL * p->sms);
  cudaError_t e = launch(tc::tc_phase_kernel<kPlanOp>, dim3(blocks), 256, 0, st, pdl, p->W, p->H, p->Kf,
                         (const float *)s.phi, p->u_hi, p->u_lo, s.acc_clear, 2 * s.M);
  if (e != cudaSuccess) return e;
  ++*kernels;
  tc::GemmArgs g = {};
  g.rows = p->H;
  g.cols = 2 * p->M;
  g.k_chunks = p->Kf / kSliceK;
  g.chunks_per_split = p->fwd_cps;
  g.limit_ns = s.limit_ns;
  g.err = s.err;
  g.W = p->W;
  g.H = p->H;
  g.Kf = p->Kf;
  g.M = p->M;
  g.Yc = p->Yc;
  g.acc_out = s.acc_out;
  g.fx_scale = s.fx_scale;
  const dim3 grid(p->rows_f / p->bn_fwd, p->rows_h / tc::kBM, p->fwd_splits);
  e = launch_gemm_bn<tc::kEpiFwd>(p->bn_fwd, p->fwd, g, grid, st, chain);
  if (e == cudaSuccess) ++*kernels;
  return e;
}

cudaError_t launch_iteration(Plan *p, const Step &s, cudaStream_t st, bool pdl, bool chain, int *kernels) {
  *kernels = 0;
  tc::PrepArgs pa = {};
  pa.H = p->H;
  pa.M = p->M;
  pa.Kb = p->Kb;
  pa.acc_in = s.acc_in;
  pa.acc_clear = s.acc_clear;
  pa.w_in = s.w_in;
  pa.w_out = s.w_out;
  pa.YT = p->YT;
  pa.p_hi = p->p_hi;
  pa.p_lo = p->p_lo;
  pa.inv_fx_n = s.inv_fx_n;
  pa.trace = s.trace;
  // blocks take even shares of the rows (each block also forms all M coefficients)
  const long long pairs = (long long)p->H * (p->Kb / 2);
  const int prep_blocks =
      (int)std::max<long long>(1, std::min<long long>({(pairs + 255) / 256, 2LL * p->sms, (long long)p->H}));
  cudaError_t e = launch(tc::tc_prep_kernel<kPlanOp>, dim3(prep_blocks), tc::kPrepThreads,
                         (int)(sizeof(float2) * p->M), st, pdl, pa);
  if (e != cudaSuccess) return e;
  ++*kernels;
  tc::GemmArgs g = {};
  g.rows = p->H;
  g.cols = 2 * p->W;
  g.k_chunks = p->Kb / kSliceK;
  g.chunks_per_split = g.k_chunks;
  g.limit_ns = s.limit_ns;
  g.err = s.err;
  g.W = p->W;
  g.H = p->H;
  g.Kf = p->Kf;
  g.phi = s.phi;
  g.u_hi = p->u_hi;
  g.u_lo = p->u_lo;
  const dim3 grid_b(p->rows_b / p->bn_back, p->rows_h / tc::kBM, 1);
  e = launch_gemm_bn<tc::kEpiBack>(p->bn_back, p->back, g, grid_b, st, chain);
  if (e != cudaSuccess) return e;
  ++*kernels;
  g = {};
  g.rows = p->H;
  g.cols = 2 * p->M;
  g.k_chunks = p->Kf / kSliceK;
  g.chunks_per_split = p->fwd_cps;
  g.limit_ns = s.limit_ns;
  g.err = s.err;
  g.W = p->W;
  g.H = p->H;
  g.Kf = p->Kf;
  g.M = p->M;
  g.Yc = p->Yc;
  g.acc_out = s.acc_out;
  g.fx_scale = s.fx_scale;
  const dim3 grid_f(p->rows_f / p->bn_fwd, p->rows_h / tc::kBM, p->fwd_splits);
  e = launch_gemm_bn<tc::kEpiFwd>(p->bn_fwd, p->fwd, g, grid_f, st, chain);
  if (e == cudaSuccess) ++*kernels;
  return e;
}

namespace {

template <int OP>
cudaError_t gemm_op(int rows, int cols, int K, const float *A, const float *B, float *C, int tile_n, cudaStream_t st,
                    int *timed_out, const char **what) {
  *timed_out = 0;
  constexpr int sk = tc::slice_k<OP>();
  const int Kp = round_up(K, sk), ra = round_up(rows, tc::kBM), rb = round_up(cols, tile_n);
  void *buf[4] = {nullptr, nullptr, nullptr, nullptr};
  int *err = nullptr;
  *what = "allocating the GEMM operands";
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 4 && e == cudaSuccess; i++)
    e = alloc_bytes(&buf[i], (size_t)(i < 2 ? ra : rb) * Kp * tc::Op<OP>::kBytes);
  if (e == cudaSuccess) e = alloc(&err, 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    *what = "splitting the GEMM operands";
    const long long ta = (long long)ra * Kp, tb = (long long)rb * Kp;
    e = launch(tc::tc_split_kernel<OP>, dim3((int)std::min<long long>((ta + 255) / 256, 4096)), 256, 0, st, false, A,
               rows, K, Kp, ta, buf[0], buf[1]);
    if (e == cudaSuccess)
      e = launch(tc::tc_split_kernel<OP>, dim3((int)std::min<long long>((tb + 255) / 256, 4096)), 256, 0, st, false, B,
                 cols, K, Kp, tb, buf[2], buf[3]);
  }
  tc::Maps maps{};
  if (e == cudaSuccess) {
    *what = "encoding the GEMM tensor maps";
    e = encode<OP>(&maps.a_hi, buf[0], Kp, ra, tc::kBM);
    if (e == cudaSuccess) e = encode<OP>(&maps.a_lo, buf[1], Kp, ra, tc::kBM);
    if (e == cudaSuccess) e = encode<OP>(&maps.b_hi, buf[2], Kp, rb, tile_n);
    if (e == cudaSuccess) e = encode<OP>(&maps.b_lo, buf[3], Kp, rb, tile_n);
  }
  if (e == cudaSuccess) {
    *what = "running the GEMM";
    tc::GemmArgs g = {};
    g.rows = rows;
    g.cols = cols;
    g.k_chunks = Kp / sk;
    g.chunks_per_split = g.k_chunks;
    g.limit_ns = 2000000000LL;
    g.err = err;
    g.C = C;
    const dim3 grid(rb / tile_n, ra / tc::kBM, 1);
    if (tile_n == 32) {
      e = set_smem<32, tc::kEpiPlain, OP>();
      if (e == cudaSuccess) e = launch_gemm<32, tc::kEpiPlain, OP>(maps, g, grid, st, false);
    } else if (tile_n == 256) {
      e = set_smem<256, tc::kEpiPlain, OP>();
      if (e == cudaSuccess) e = launch_gemm<256, tc::kEpiPlain, OP>(maps, g, grid, st, false);
    } else if (tile_n == 128) {
      e = set_smem<128, tc::kEpiPlain, OP>();
      if (e == cudaSuccess) e = launch_gemm<128, tc::kEpiPlain, OP>(maps, g, grid, st, false);
    } else {
      e = set_smem<64, tc::kEpiPlain, OP>();
      if (e == cudaSuccess) e = launch_gemm<64, tc::kEpiPlain, OP>(maps, g, grid, st, false);
    }
  }
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, err, sizeof flag, cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  *timed_out = flag;
  for (void *b : buf)
    if (b) cudaFree(b);
  if (err) cudaFree(err);
  return e;
}

}  // namespace

cudaError_t gemm(int rows, int cols, int K, const float *A, const float *B, float *C, int tile_n, int operands,
                 cudaStream_t st, int *timed_out, const char **what) {
  return operands == 1 ? gemm_op<tc::kOpF16>(rows, cols, K, A, B, C, tile_n, st, timed_out, what)
                       : gemm_op<tc::kOpTF32>(rows, cols, K, A, B, C, tile_n, st, timed_out, what);
}

}  // namespace hot_tc
