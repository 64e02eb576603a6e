// hot.cu -- host runtime and C ABI (include/hot.h) of the GSW hologram engine.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <iterator>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/hot.h"
#include "gsw_kernels.cuh"
#include "once.h"
#include "tc.h"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

#define HOT_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? HOT_ENOMEM : HOT_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                   \
  } while (0)

template <typename T>
int dalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) return HOT_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? HOT_ENOMEM : HOT_ECUDA, "cudaMalloc(%zu B): %s",
                count * sizeof(T), cudaGetErrorString(e));
  }
  return HOT_OK;
}

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

}  // namespace

struct hot_ctx {
  int W = 0, H = 0;
  int H_total = 0, y_off = 0;  // row band: rows y_off .. y_off+H-1 of a W x H_total hologram
  double pitch = 0, lam = 0, focal = 0;
  cudaStream_t st = nullptr;
  int dev = 0;
  int precision = HOT_PREC_ACCURATE;
  // work schedule of the step kernels (see hot::SubTile)
  int grid = 0, n_sub = 0;
  hot::SubTile *sub = nullptr;  // [n_sub]
  int *first = nullptr;         // [grid + 1]
  int sched_smem_M = -1;        // M the schedule's occupancy was computed for
  // tiling (hot_set_tiling): rows per sub-tile (pixels per thread), resident blocks per SM
  // (0: as many as fit), traps per staged chunk
  int tile_rows = hot::kRowsMax, tile_bps = 0, tile_chunk = hot::kChunk;
  int sched_bps = 0, sched_bps_max = 0;  // resident blocks per SM in the schedule; occupancy limit
  int tile_merge = 1;  // hot_set_block_merge: schedule blocks per launched block of the GSW step (1, 2, 4)
  int groups = 1;      // schedule blocks per launched block of the direct GSW step (1 or 4)
  // one-exponential step of the direct modes (hot_set_once; M <= hot::kOnceMaxM): requested,
  // shape in effect (hot::once_shape; 0: the direct step kernels) and its own schedule
  bool once_req = true;
  int once = 0;
  hot::SubTile *osub = nullptr;  // [on_sub]
  int *ofirst = nullptr;         // [ogrid + 1]
  int ogrid = 0, on_sub = 0;
  // the same block runs cut into sub-tiles of hot::kOnceFwdRows rows: the forward field of given phases
  hot::SubTile *ofsub = nullptr;
  int *offirst = nullptr;
  // the unit phasors u_j = S_j/|S_j| of phi, written by the last step of a one-exponential hot_gsw
  // (hot::StepArgs::u_out); valid while phi is the phases that step wrote.  The next hot_gsw's first
  // forward field then reads them (gsw_from_u) and so adds the terms an uninterrupted run adds.
  float2 *ubuf = nullptr;  // [N]
  bool u_valid = false, gsw_from_u = false;
  int shard_k = -1;                      // last launch of a sharded sequence (hot_sharded_*)
  // state
  float *phi = nullptr;  // [N]
  int M = 0;
  double *abc = nullptr;                                       // [M][3]
  float *Xt = nullptr, *Yt = nullptr, *Xr = nullptr, *Yr = nullptr;  // tables
  float *Y4t = nullptr, *Y4r = nullptr;  // [4][M][ldy4] shifted row tables (hot::StepArgs::Y4)
  int ldy4 = 0;
  float2 *Xc = nullptr, *Yc = nullptr;                               // complex tables (separable)
  float2 *Yc2 = nullptr;  // [2][M][ldy4] row-shifted copies of Yc (hot::StepArgs::Yc)
  float *w = nullptr;                                          // [2][M] weights (home: w[0])
  unsigned long long *acc = nullptr;                           // [3][copies][2][M] fixed-point field sums
  long long *Vsum = nullptr;                                   // [2][M] sums of the last forward
  float *metrics = nullptr;                                    // [2]
  int fx_shift = 0;                                            // fixed-point scale 2^fx_shift
  unsigned char *u8 = nullptr;                                 // [N] staging for host output
  bool have_fields = false;
  long long launches = 0;
  // instrumentation
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  bool profiling = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> spare;
  // CUDA graphs of whole hot_gsw(iters) launch sequences, keyed by (iters, precision)
  struct Graph {
    int iters, precision;
    bool from_u;  // the first forward field reads ubuf
    long long kernels;
    cudaGraphExec_t exec;
  };
  bool use_graphs = true;
  cudaStream_t cap = nullptr;  // capture stream (capture is not allowed on the legacy stream)
  // persistent form (one cooperative launch per hot_gsw): grid barrier state [count, gen, err]
  bool persistent = false;
  // convergence trace (hot_set_trace): e, u of the field read by each iteration of hot_gsw
  bool tracing = false;
  float *trace = nullptr;  // [trace_cap][2]
  int trace_cap = 0, trace_iters = -1;
  double wait_limit_s = 2.0;
  unsigned int *sync = nullptr;
  std::vector<Graph> graphs;
  // HOT_PREC_TENSOR: operands and launch shapes of the tensor-core iteration (built on first use)
  hot_tc::Plan *tc = nullptr;
  float2 *G = nullptr;  // [M] adjoint coefficients of hot_intensity_loss (allocated on first use)
};

namespace {

bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

// Copies of each fixed-point accumulator buffer (StepArgs::copies).  With few traps all blocks
// add into the same 2M addresses at nearly the same moment; 8 copies (block b adds into copy
// b % 8) spread those atomics.  The separable kernel reads the copies; the direct kernels,
// whose registers are fully used, keep one.  Storage is sized for the largest count.
int acc_copies(const hot_ctx *c) { return (c->precision == HOT_PREC_SEPARABLE && c->M <= 512) ? 8 : 1; }

// Modes whose step kernels are the separable ones: HOT_PREC_SEPARABLE, and HOT_PREC_TENSOR for
// every launch outside the GSW loop (forward field and adjoint of given phases, superposition).
bool separable_kernels(const hot_ctx *c) {
  return c->precision == HOT_PREC_SEPARABLE || c->precision == HOT_PREC_TENSOR;
}
size_t acc_elems(int M) { return 6 * (size_t)M * (M <= 512 ? 8 : 1); }

// Pixels of the whole hologram (all row bands): the normalisation 1/N of Eq. 1.
double n_total(const hot_ctx *c) { return (double)c->W * (double)c->H_total; }

// Fixed-point scale of the field sums: |sum| <= N (whole hologram), kept below 2^61.
int fixed_point_shift(long long n) {
  int bits = 0;
  while ((1LL << bits) < n) bits++;
  return 61 - bits;
}

void drop_graphs(hot_ctx *c) {
  for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

void free_traps(hot_ctx *c) {
  drop_graphs(c);
  hot_tc::plan_destroy(c->tc);
  c->tc = nullptr;
  dfree(c->abc);
  dfree(c->Xt);
  dfree(c->Yt);
  dfree(c->Xr);
  dfree(c->Yr);
  dfree(c->Y4t);
  dfree(c->Y4r);
  dfree(c->Xc);
  dfree(c->Yc);
  dfree(c->Yc2);
  dfree(c->w);
  dfree(c->acc);
  dfree(c->Vsum);
  dfree(c->G);
  c->M = 0;
  c->have_fields = false;
  c->u_valid = false;
}

int check_launch(hot_ctx *c, const char *what) {
  c->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(HOT_ECUDA, "launch of %s: %s", what, cudaGetErrorString(e));
  return HOT_OK;
}

cudaEvent_t take_event(hot_ctx *c) {
  if (!c->spare.empty()) {
    cudaEvent_t e = c->spare.back();
    c->spare.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void clear_records(hot_ctx *c) {
  for (auto &r : c->recs) {
    c->spare.push_back(r.a);
    c->spare.push_back(r.b);
  }
  c->recs.clear();
}

// Brackets one kernel launch with events when profiling is on.
struct Probe {
  hot_ctx *c;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  Probe(hot_ctx *ctx, int k) : c(ctx), kind(k) {
    if (!c->profiling) return;
    a = take_event(c);
    b = take_event(c);
    if (a && b) cudaEventRecord(a, c->st);
  }
  ~Probe() {
    if (!a || !b) return;
    cudaEventRecord(b, c->st);
    c->recs.push_back({kind, a, b});
  }
};

// Launches kernel<<<grid, block, smem, c->st>>>(args...); with pdl, as a programmatic
// dependent of the previous kernel in the stream (its prologue may overlap that kernel).
template <typename... KArgs, typename... Args>
void launch(hot_ctx *c, void (*kernel)(KArgs...), int grid, int block, int smem, bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Launch k of a hot_gsw sequence (k = 0: forward field of the starting phases; k >= 1:
// iteration k).  Accumulators rotate over three buffers, weights over two.
hot::StepArgs make_step_args(const hot_ctx *c, int k, const float *phi, const float2 *G, float *grad) {
  const bool fast = c->precision == HOT_PREC_FAST;
  hot::StepArgs a = {};
  a.W = c->W;
  a.H = c->H;
  a.M = c->M;
  a.chunk = c->tile_chunk;
  a.sub = c->sub;
  a.first = c->first;
  a.X = fast ? c->Xr : c->Xt;
  a.Y = fast ? c->Yr : c->Yt;
  a.Y4 = fast ? c->Y4r : c->Y4t;
  a.ldy4 = c->ldy4;
  a.Xc = c->Xc;
  a.Yc = c->Yc2;
  a.phi = c->phi;
  const size_t M2 = 2 * (size_t)c->M * acc_copies(c);
  a.copies = acc_copies(c);
  a.acc_in = c->acc + M2 * ((k + 2) % 3);
  a.acc_out = c->acc + M2 * (k % 3);
  a.acc_clear = c->acc + M2 * ((k + 1) % 3);
  a.w_in = c->w + (size_t)c->M * ((k + 1) & 1);
  a.w_out = c->w + (size_t)c->M * (k & 1);
  a.fx_scale = ldexpf(1.0f, c->fx_shift);
  a.inv_fx_n = (float)(1.0 / (n_total(c) * ldexp(1.0, c->fx_shift)));
  a.angle_units = fast ? 1.0f : 0.15915494309189535f;
  a.angle_eta = fast ? hot::kFastEta : 0.0f;
  if (phi) a.phi = const_cast<float *>(phi);  // read only: forward field or adjoint of given phases
  a.G = G;
  a.grad = grad;
  a.inv_n = (float)(1.0 / (n_total(c)));
  a.trace = (c->tracing && c->trace && k >= 1 && k <= c->trace_cap) ? c->trace + 2 * (k - 1) : nullptr;
  a.once_flags = 0;
  return a;
}

// Traps staged at once by the separable kernel (its shared memory is sized by it).
int sep_chunk(const hot_ctx *c) { return std::max(1, std::min(c->M, c->tile_chunk)); }

template <bool FAST, bool BACK, bool FWD, bool ADJ = false>
int launch_tile(hot_ctx *c, bool pdl, int k, const float *phi = nullptr, const float2 *G = nullptr,
                float *grad = nullptr) {
  const hot::StepArgs a = make_step_args(c, k, phi, G, grad);
  const int smem = hot::step_smem_bytes(c->M, BACK);
  Probe p(c, BACK && FWD ? HOT_KERNEL_STEP : FWD ? HOT_KERNEL_FORWARD : HOT_KERNEL_OTHER);
  if (BACK && FWD && !ADJ && c->groups == 4)  // the GSW step, merged: one block per SM
    launch(c, hot::gsw_step_kernel<FAST, true, true, false, 4>, c->grid / 4, hot::kThreads * 4, smem * 4, pdl, a);
  else if (BACK && FWD && !ADJ && c->groups == 2)  // two blocks per SM, two schedule blocks each
    launch(c, hot::gsw_step_kernel<FAST, true, true, false, 2>, c->grid / 2, hot::kThreads * 2, smem * 2, pdl, a);
  else
    launch(c, hot::gsw_step_kernel<FAST, BACK, FWD, ADJ>, c->grid, hot::kThreads, smem, pdl, a);
  return check_launch(c, "gsw_step_kernel");
}

template <bool BACK, bool FWD, bool ADJ = false>
int launch_sep(hot_ctx *c, bool pdl, int k, const float *phi = nullptr, const float2 *G = nullptr,
               float *grad = nullptr) {
  hot::StepArgs a = make_step_args(c, k, phi, G, grad);
  a.chunk = sep_chunk(c);
  Probe p(c, BACK && FWD ? HOT_KERNEL_STEP : FWD ? HOT_KERNEL_FORWARD : HOT_KERNEL_OTHER);
  launch(c, hot::gsw_sep_kernel<BACK, FWD, ADJ>, c->grid, hot::kThreads, hot::sep_smem_bytes(a.chunk), pdl, a);
  return check_launch(c, "gsw_sep_kernel");
}

// The one-exponential step (BACK: weight update, back-projection and forward field) or its
// forward field of given phases, on the context's one-exponential schedule.
template <bool BACK>
int launch_once(hot_ctx *c, bool pdl, int k, const float *phi, bool last) {
  hot::StepArgs a = make_step_args(c, k, phi, nullptr, nullptr);
  a.u = c->ubuf;
  a.once_flags = (last ? hot::kOnceLast : 0) | (!BACK && !phi && c->gsw_from_u ? hot::kOnceReadU : 0);
  a.sub = BACK ? c->osub : c->ofsub;
  a.first = BACK ? c->ofirst : c->offirst;
  a.chunk = c->M;
  Probe p(c, BACK ? HOT_KERNEL_STEP : HOT_KERNEL_FORWARD);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->ogrid);
  cfg.blockDim = dim3(hot::kThreads);
  cfg.stream = c->st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  hot_once::launch_step(c->once, c->precision == HOT_PREC_FAST, BACK, cfg, a);
  return check_launch(c, "gsw_once_kernel");
}

// The step kernel of the context's mode (accurate / fast direct evaluation, or separable).
template <bool BACK, bool FWD, bool ADJ = false>
int launch_mode(hot_ctx *c, bool pdl, int k, const float *phi = nullptr, const float2 *G = nullptr,
                float *grad = nullptr, bool last = true) {
  if (separable_kernels(c)) return launch_sep<BACK, FWD, ADJ>(c, pdl, k, phi, G, grad);
  if (c->once && FWD && !ADJ && !G) {
    // the forward field a call opens with, of phases the caller set: the separable kernel
    // (complex tables, FMA only) at about half the cost of evaluating every exponential
    if (!BACK && !phi && !c->gsw_from_u) return launch_sep<false, true>(c, pdl, k);
    return launch_once<BACK>(c, pdl, k, phi, last);
  }
  if (c->precision == HOT_PREC_FAST) return launch_tile<true, BACK, FWD, ADJ>(c, pdl, k, phi, G, grad);
  return launch_tile<false, BACK, FWD, ADJ>(c, pdl, k, phi, G, grad);
}

// Raises the dynamic shared-memory limit of every step-kernel variant to what M needs.
int set_step_smem(int M) {
  const int back = hot::step_smem_bytes(M, true), fwd = hot::step_smem_bytes(M, false);
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, back));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, back));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, back));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, back));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fwd));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fwd));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<true, true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, back));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<false, true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, back));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<true, true, true, false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * back));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<false, true, true, false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * back));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<true, true, true, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * back));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<false, true, true, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * back));
  const int sep = hot::sep_smem_bytes(hot::kChunk);
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_sep_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sep));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_sep_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sep));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_sep_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sep));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_sep_kernel<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sep));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_persistent_kernel<hot::kModeAccurate>, cudaFuncAttributeMaxDynamicSharedMemorySize, back));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_persistent_kernel<hot::kModeFast>, cudaFuncAttributeMaxDynamicSharedMemorySize, back));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_persistent_kernel<hot::kModeSeparable>, cudaFuncAttributeMaxDynamicSharedMemorySize, sep));
  return HOT_OK;
}

// The W/32 x H row segments dealt out to G blocks in equal contiguous runs (to within one
// segment), each run cut into sub-tiles of at most `rows` rows -- evenly, or (full) into
// sub-tiles of exactly `rows` rows and one shorter remainder; block b walks sub-tiles
// first[b] .. first[b + 1] - 1.
void cut_schedule(int W, int H, int G, int rows, std::vector<hot::SubTile> &sub, std::vector<int> &first,
                  bool full = false) {
  const int strips = (W + hot::kTileW - 1) / hot::kTileW;
  const long long U = (long long)strips * H;
  sub.clear();
  first.assign(G + 1, 0);
  for (int b = 0; b < G; b++) {
    first[b] = (int)sub.size();
    long long s = U * b / G;
    const long long s1 = U * (b + 1) / G;
    while (s < s1) {
      const int strip = (int)(s / H), row = (int)(s % H);
      const long long run_end = std::min<long long>(s1, (long long)(strip + 1) * H);
      const int L = (int)(run_end - s);
      const int nsub = (L + rows - 1) / rows;
      for (int i = 0; i < nsub; i++) {
        const int r0 = row + (full ? i * rows : (int)((long long)L * i / nsub));
        const int r1 = full ? std::min(r0 + rows, row + L) : row + (int)((long long)L * (i + 1) / nsub);
        sub.push_back({strip * hot::kTileW, r0, r1 - r0, 0});
      }
      s = run_end;
    }
  }
  first[G] = (int)sub.size();
}

// The one-exponential step's schedule (one wave of its blocks, sub-tiles of its R rows), when
// the context's mode and trap count allow it and it is requested; otherwise c->once = 0.
int build_once_schedule(hot_ctx *c, int sms) {
  c->once = 0;
  c->ogrid = 0;
  c->on_sub = 0;
  dfree(c->osub);
  dfree(c->ofirst);
  dfree(c->ofsub);
  dfree(c->offirst);
  const int shape = hot::once_shape(c->M);
  if (!c->once_req || !shape || (c->precision != HOT_PREC_FAST && c->precision != HOT_PREC_ACCURATE)) return HOT_OK;
  int per_sm = 0, rc = HOT_OK;
  HOT_CUDA(hot_once::occupancy(shape, &per_sm));
  if (per_sm < 1) return HOT_OK;  // no room: the direct kernels
  const long long U = (long long)((c->W + hot::kTileW - 1) / hot::kTileW) * c->H;
  const int G = (int)std::min<long long>((long long)sms * per_sm, U);
  std::vector<hot::SubTile> sub;
  std::vector<int> first;
  std::vector<hot::SubTile> fsub;
  std::vector<int> ffirst;
  cut_schedule(c->W, c->H, G, hot::once_rows(shape), sub, first, true);
  cut_schedule(c->W, c->H, G, hot::kOnceFwdRows, fsub, ffirst, true);
  rc = dalloc(&c->osub, sub.size());
  if (rc == HOT_OK) rc = dalloc(&c->ofirst, first.size());
  if (rc == HOT_OK) rc = dalloc(&c->ofsub, fsub.size());
  if (rc == HOT_OK) rc = dalloc(&c->offirst, ffirst.size());
  if (rc != HOT_OK) return rc;
  HOT_CUDA(cudaMemcpy(c->osub, sub.data(), sizeof(hot::SubTile) * sub.size(), cudaMemcpyHostToDevice));
  HOT_CUDA(cudaMemcpy(c->ofirst, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice));
  HOT_CUDA(cudaMemcpy(c->ofsub, fsub.data(), sizeof(hot::SubTile) * fsub.size(), cudaMemcpyHostToDevice));
  HOT_CUDA(cudaMemcpy(c->offirst, ffirst.data(), sizeof(int) * ffirst.size(), cudaMemcpyHostToDevice));
  if (!c->ubuf) {
    rc = dalloc(&c->ubuf, (size_t)c->W * c->H);
    if (rc != HOT_OK) return rc;
  }
  c->ogrid = G;
  c->on_sub = (int)sub.size();
  c->once = shape;
  return HOT_OK;
}

// One wave of persistent blocks (SMs x resident blocks per SM: as many as fit, at most
// tile_bps); the W/32 x H row segments are dealt out in equal contiguous runs, cut into
// sub-tiles of <= tile_rows rows.  Also the one-exponential step's schedule.
int build_schedule(hot_ctx *c) {
  drop_graphs(c);  // graphs hold the old schedule
  int rc = set_step_smem(c->M);
  if (rc != HOT_OK) return rc;
  int sms = 0, per_sm = 0;
  HOT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
  // the per-iteration and the persistent kernels share the schedule (so that they compute the
  // same bits): as many blocks per SM as both can keep resident
  int per_sm_p = 0;
  if (separable_kernels(c)) {
    const int smem = hot::sep_smem_bytes(sep_chunk(c));
    HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hot::gsw_sep_kernel<true, true>, hot::kThreads, smem));
    HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_p, hot::gsw_persistent_kernel<hot::kModeSeparable>,
                                                           hot::kThreads, smem));
  } else {
    const int smem = hot::step_smem_bytes(c->M, true);
    HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hot::gsw_step_kernel<true, true, true>,
                                                           hot::kThreads, smem));
    HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_p, hot::gsw_persistent_kernel<hot::kModeFast>,
                                                           hot::kThreads, smem));
    int per_sm_a = 0;
    HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_a, hot::gsw_persistent_kernel<hot::kModeAccurate>,
                                                           hot::kThreads, smem));
    per_sm_p = std::min(per_sm_p, per_sm_a);
  }
  per_sm = std::min(per_sm, per_sm_p);
  if (per_sm < 1) per_sm = 1;
  c->sched_bps_max = per_sm;
  if (c->tile_bps > 0 && c->tile_bps < per_sm) per_sm = c->tile_bps;
  c->sched_bps = per_sm;
  // Merged (hot_set_block_merge), with four schedule blocks per SM the direct modes' GSW step
  // runs one block per SM holding four of them (see gsw_step_kernel), if such a block fits.
  c->groups = 1;
  if (c->tile_merge > 1 && !separable_kernels(c) && per_sm == hot::kMaxGroups) {
    int per_sm_g = 0;
    const int smem = c->tile_merge * hot::step_smem_bytes(c->M, true);
    if (c->tile_merge == 4)
      HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_g, hot::gsw_step_kernel<true, true, true, false, 4>,
                                                             hot::kThreads * 4, smem));
    else
      HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_g, hot::gsw_step_kernel<true, true, true, false, 2>,
                                                             hot::kThreads * 2, smem));
    if (per_sm_g * c->tile_merge >= per_sm) c->groups = c->tile_merge;
  }
  const int strips = (c->W + hot::kTileW - 1) / hot::kTileW;
  const long long U = (long long)strips * c->H;
  int G = (int)std::min<long long>((long long)sms * per_sm, U);
  // whole merged blocks; rounded the same way unmerged, so that merging never changes the schedule
  // (and with it the bits of the results)
  if (!separable_kernels(c) && per_sm == hot::kMaxGroups) G = (G + hot::kMaxGroups - 1) / hot::kMaxGroups * hot::kMaxGroups;
  std::vector<hot::SubTile> sub;
  std::vector<int> first;
  cut_schedule(c->W, c->H, G, c->tile_rows, sub, first);
  HOT_CUDA(cudaStreamSynchronize(c->st));
  dfree(c->sub);
  dfree(c->first);
  c->grid = 0;
  c->n_sub = 0;
  rc = dalloc(&c->sub, sub.size());
  if (rc == HOT_OK) rc = dalloc(&c->first, first.size());
  if (rc != HOT_OK) return rc;
  HOT_CUDA(cudaMemcpy(c->sub, sub.data(), sizeof(hot::SubTile) * sub.size(), cudaMemcpyHostToDevice));
  HOT_CUDA(cudaMemcpy(c->first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice));
  c->grid = G;
  c->n_sub = (int)sub.size();
  return build_once_schedule(c, sms);
}

// One step-kernel launch (launch k of the sequence): weight update + back-projection and/or
// forward field.  last: the last launch of a call (the one-exponential step writes the phases only
// then; every other kernel writes them at each launch).
int launch_step(hot_ctx *c, bool back, bool fwd, bool pdl, int k, bool last = true) {
  if (back && fwd) return launch_mode<true, true>(c, pdl, k, nullptr, nullptr, nullptr, last);
  if (back) return launch_mode<true, false>(c, pdl, k);
  return launch_mode<false, true>(c, pdl, k);
}

// After the last launch (k = iters): Eq. 4 metrics, field sums, weights home, accumulators cleared.
int launch_finalize(hot_ctx *c, bool pdl, int iters) {
  hot::FinalizeArgs f = {};  // done = NULL: no completion stamp
  const size_t M2 = 2 * (size_t)c->M * acc_copies(c);
  f.M = c->M;
  f.copies = acc_copies(c);
  f.acc = c->acc + M2 * (iters % 3);
  f.acc_all = c->acc;
  f.w_src = c->w + (size_t)c->M * (iters & 1);
  f.w_dst = c->w;
  f.Vsum = c->Vsum;
  f.metrics = c->metrics;
  f.inv_fx_n = (float)(1.0 / (n_total(c) * ldexp(1.0, c->fx_shift)));
  Probe p(c, HOT_KERNEL_FINISH);
  launch(c, hot::gsw_finalize_kernel, 1, hot::kFinalizeThreads, 0, pdl, f);
  return check_launch(c, "gsw_finalize_kernel");
}

// The launch sequence of hot_gsw(iters) on c->st.
// Inside the sequence every kernel is a programmatic dependent of the one before it (except
// when profiling, where events separate the launches); the first one waits normally for
// whatever preceded hot_gsw in the stream (trap tables, phases).
// Phase tables of the context's traps (Eq. 2 split into column and row parts).
int launch_build_tables(hot_ctx *c) {
  const long long total = (long long)c->M * (c->W + c->H);
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  Probe p(c, HOT_KERNEL_OTHER);
  hot::build_tables_kernel<<<blocks, 256, 0, c->st>>>(c->W, c->H, c->H_total, c->y_off, c->M, c->abc, c->Xt, c->Yt,
                                                      c->Xr, c->Yr, c->Xc, c->Yc, c->Y4t, c->Y4r, c->ldy4, c->Yc2);
  int rc = check_launch(c, "build_tables_kernel");
  if (rc == HOT_OK && c->tc) {  // the tensor-core operands derive from the tables
    cudaError_t e = hot_tc::plan_refresh(c->tc, c->st);
    if (e != cudaSuccess) rc = fail(HOT_ECUDA, "rebuilding the tensor-core operands: %s", cudaGetErrorString(e));
    c->launches++;
  }
  return rc;
}

// The tensor-core plan of the context's traps (HOT_PREC_TENSOR), built on first use.
int ensure_tc_plan(hot_ctx *c) {
  if (c->tc) return HOT_OK;
  const char *what = "";
  cudaError_t e = hot_tc::plan_create(&c->tc, c->W, c->H, c->M, c->Xc, c->Yc, c->st, &what);
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? HOT_ENOMEM : HOT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  c->launches++;
  return HOT_OK;
}

hot_tc::Step tc_step(hot_ctx *c, int k) {
  const hot::StepArgs a = make_step_args(c, k, nullptr, nullptr, nullptr);
  hot_tc::Step s;
  s.M = c->M;
  s.acc_in = a.acc_in;
  s.acc_out = a.acc_out;
  s.acc_clear = a.acc_clear;
  s.w_in = a.w_in;
  s.w_out = a.w_out;
  s.phi = c->phi;
  s.trace = a.trace;
  s.fx_scale = a.fx_scale;
  s.inv_fx_n = a.inv_fx_n;
  s.err = reinterpret_cast<int *>(c->sync + 2);
  s.limit_ns = (long long)(c->wait_limit_s * 1e9);
  return s;
}

// Launch k of the tensor-core sequence: k = 0 the forward field of the phases, k >= 1 iteration k.
int launch_tc(hot_ctx *c, bool pdl, int k) {
  Probe p(c, k ? HOT_KERNEL_STEP : HOT_KERNEL_FORWARD);
  int kernels = 0;
  const bool chain = !c->profiling;
  const cudaError_t e = k ? hot_tc::launch_iteration(c->tc, tc_step(c, k), c->st, pdl, chain, &kernels)
                          : hot_tc::launch_forward(c->tc, tc_step(c, k), c->st, pdl, chain, &kernels);
  c->launches += kernels;
  if (e != cudaSuccess) return fail(HOT_ECUDA, "tensor-core launch %d: %s", k, cudaGetErrorString(e));
  return HOT_OK;
}

// The whole sequence of enqueue_gsw's step launches as one cooperative launch (all blocks
// resident; the grid is one wave by construction of the schedule).
int launch_persistent(hot_ctx *c, int iters) {
  hot::PersistArgs p = {};
  for (int j = 0; j < 6; j++) {
    p.step[j] = make_step_args(c, j, nullptr, nullptr, nullptr);
    if (c->precision == HOT_PREC_SEPARABLE) p.step[j].chunk = sep_chunk(c);
  }
  if (c->once)
    for (int j = 0; j < 6; j++) p.step[j].u = c->ubuf;
  p.step[0].once_flags = c->gsw_from_u ? hot::kOnceReadU : 0;  // launch 0: the forward field of phi
  p.k0 = 0;
  p.iters = iters;
  p.trace = c->tracing ? c->trace : nullptr;
  p.sync.count = c->sync;
  p.sync.err = reinterpret_cast<int *>(c->sync + 2);
  p.sync.limit_ns = (long long)(c->wait_limit_s * 1e9);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->grid);
  cfg.blockDim = dim3(hot::kThreads);
  cfg.stream = c->st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  HOT_CUDA(cudaMemsetAsync(c->sync, 0, sizeof(unsigned int), c->st));  // arrival count
  Probe probe(c, HOT_KERNEL_STEP);
  if (c->once) {
    if (!c->gsw_from_u) {  // launch 0 as in enqueue_gsw: the separable forward field of phi
      const int rc = launch_sep<false, true>(c, false, 0);
      if (rc != HOT_OK) return rc;
      p.k0 = 1;
    }
    for (int j = 0; j < 6; j++) {
      p.step[j].sub = c->osub;
      p.step[j].first = c->ofirst;
      p.step[j].chunk = c->M;
    }
    cfg.gridDim = dim3(c->ogrid);
    hot_once::launch_persistent(c->once, c->precision == HOT_PREC_FAST, cfg, p);
  } else if (c->precision == HOT_PREC_SEPARABLE) {
    cfg.dynamicSmemBytes = hot::sep_smem_bytes(sep_chunk(c));
    cudaLaunchKernelEx(&cfg, hot::gsw_persistent_kernel<hot::kModeSeparable>, p);
  } else if (c->precision == HOT_PREC_FAST) {
    cfg.dynamicSmemBytes = hot::step_smem_bytes(c->M, true);
    cudaLaunchKernelEx(&cfg, hot::gsw_persistent_kernel<hot::kModeFast>, p);
  } else {
    cfg.dynamicSmemBytes = hot::step_smem_bytes(c->M, true);
    cudaLaunchKernelEx(&cfg, hot::gsw_persistent_kernel<hot::kModeAccurate>, p);
  }
  return check_launch(c, "gsw_persistent_kernel");
}

// Reads the barrier's error flag (synchronises): after a wait ran out, the accumulators and the
// barrier are reset and HOT_ETIMEOUT is returned; the phases are then undefined.
int check_wait_error(hot_ctx *c, const char *who) {
  unsigned int st[3] = {0, 0, 0};  // [2]: error flag of the bounded waits
  HOT_CUDA(cudaMemcpyAsync(st, c->sync, sizeof st, cudaMemcpyDeviceToHost, c->st));
  HOT_CUDA(cudaStreamSynchronize(c->st));
  if (!st[2]) return HOT_OK;
  HOT_CUDA(cudaMemsetAsync(c->sync, 0, sizeof st, c->st));
  if (c->M) HOT_CUDA(cudaMemsetAsync(c->acc, 0, sizeof(unsigned long long) * acc_elems(c->M), c->st));
  HOT_CUDA(cudaStreamSynchronize(c->st));
  c->have_fields = false;
  c->u_valid = false;
  return fail(HOT_ETIMEOUT, "%s: a bounded device-side wait ran out (limit %.3g s)", who, c->wait_limit_s);
}

int enqueue_gsw(hot_ctx *c, int iters) {
  if (c->persistent) {
    int rc = launch_persistent(c, iters);
    if (rc == HOT_OK) rc = launch_finalize(c, false, iters);
    return rc;
  }
  const bool pdl = !c->profiling;
  if (c->precision == HOT_PREC_TENSOR) {
    int rc = launch_tc(c, false, 0);
    for (int k = 1; k <= iters && rc == HOT_OK; k++) rc = launch_tc(c, pdl, k);
    if (rc == HOT_OK) rc = launch_finalize(c, pdl, iters);
    return rc;
  }
  int rc = launch_step(c, false, true, false, 0);       // V^1 = F(phi^0)
  for (int k = 1; k <= iters && rc == HOT_OK; k++)      // w^k, c^k from V^k; phi^k; V^{k+1} = F(phi^k)
    rc = launch_step(c, true, true, pdl, k, k == iters);
  if (rc == HOT_OK) rc = launch_finalize(c, pdl, iters);  // e, u of V^{iters+1}
  return rc;
}

// Replays (capturing on first use) the graph of enqueue_gsw(iters).
int launch_gsw_graph(hot_ctx *c, int iters) {
  for (auto &g : c->graphs)
    if (g.iters == iters && g.precision == c->precision && g.from_u == c->gsw_from_u) {
      HOT_CUDA(cudaGraphLaunch(g.exec, c->st));
      c->launches += g.kernels;
      return HOT_OK;
    }
  if (!c->cap) HOT_CUDA(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  if (c->graphs.size() >= 8) {
    cudaGraphExecDestroy(c->graphs.front().exec);
    c->graphs.erase(c->graphs.begin());
  }
  cudaStream_t user = c->st;
  const long long before = c->launches;
  HOT_CUDA(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  c->st = c->cap;
  int rc = enqueue_gsw(c, iters);
  c->st = user;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &graph);
  const long long kernels = c->launches - before;
  c->launches = before;
  if (rc != HOT_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(HOT_ECUDA, "hot_gsw: graph capture: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(HOT_ECUDA, "hot_gsw: graph instantiation: %s", cudaGetErrorString(e));
  c->graphs.push_back({iters, c->precision, c->gsw_from_u, kernels, exec});
  HOT_CUDA(cudaGraphLaunch(exec, c->st));
  c->launches += kernels;
  return HOT_OK;
}

}  // namespace

extern "C" {

const char *hot_last_error(void) { return g_err; }

int hot_create(hot_ctx **out, int width, int height, double pitch_m, double wavelength_m,
               double focal_m, void *cuda_stream) {
  g_err[0] = 0;
  if (!out) return fail(HOT_EINVAL, "hot_create: out is NULL");
  *out = nullptr;
  if (width < 1 || height < 1 || (long long)width * height >= (1LL << 31))
    return fail(HOT_EINVAL, "hot_create: invalid size %d x %d", width, height);
  if (!finite_pos(pitch_m) || !finite_pos(wavelength_m) || !finite_pos(focal_m))
    return fail(HOT_EINVAL, "hot_create: pitch, wavelength and focal length must be finite and > 0");
  hot_ctx *c = new (std::nothrow) hot_ctx;
  if (!c) return fail(HOT_ENOMEM, "hot_create: out of host memory");
  c->W = width;
  c->H = height;
  c->pitch = pitch_m;
  c->lam = wavelength_m;
  c->focal = focal_m;
  c->st = static_cast<cudaStream_t>(cuda_stream);
  c->H_total = height;
  c->fx_shift = fixed_point_shift((long long)width * height);
  int rc = HOT_OK;
  cudaError_t e = cudaGetDevice(&c->dev);
  if (e != cudaSuccess) rc = fail(HOT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  const size_t N = (size_t)width * height;
  if (rc == HOT_OK) rc = dalloc(&c->phi, N);
  if (rc == HOT_OK) rc = dalloc(&c->metrics, 2);
  if (rc == HOT_OK) rc = dalloc(&c->sync, 3);
  if (rc == HOT_OK && cudaMemsetAsync(c->sync, 0, 3 * sizeof(unsigned int), c->st) != cudaSuccess)
    rc = fail(HOT_ECUDA, "hot_create: clearing the barrier state failed");
  if (rc == HOT_OK) {
    e = cudaMemsetAsync(c->phi, 0, N * sizeof(float), c->st);
    if (e != cudaSuccess) rc = fail(HOT_ECUDA, "hot_create: %s", cudaGetErrorString(e));
  }
  if (rc != HOT_OK) {
    hot_destroy(c);
    return rc;
  }
  *out = c;
  return HOT_OK;
}

void hot_destroy(hot_ctx *c) {
  if (!c) return;
  if (c->phi || c->M) cudaStreamSynchronize(c->st);
  drop_graphs(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  clear_records(c);
  for (cudaEvent_t e : c->spare) cudaEventDestroy(e);
  c->spare.clear();
  free_traps(c);
  dfree(c->phi);
  dfree(c->sub);
  dfree(c->first);
  dfree(c->osub);
  dfree(c->ofirst);
  dfree(c->ofsub);
  dfree(c->offirst);
  dfree(c->ubuf);
  dfree(c->metrics);
  dfree(c->u8);
  dfree(c->sync);
  dfree(c->trace);
  delete c;
}

int hot_set_traps(hot_ctx *c, int M, const double *xyz_m, const double *w0) {
  if (!c) return fail(HOT_EINVAL, "hot_set_traps: NULL context");
  if (M < 1 || M > HOT_MAX_TRAPS) return fail(HOT_EINVAL, "hot_set_traps: M = %d not in [1, %d]", M, HOT_MAX_TRAPS);
  if (!xyz_m) return fail(HOT_EINVAL, "hot_set_traps: xyz is NULL");
  for (int i = 0; i < 3 * M; i++)
    if (!std::isfinite(xyz_m[i])) return fail(HOT_EINVAL, "hot_set_traps: coordinate %d not finite", i);
  if (w0)
    for (int m = 0; m < M; m++)
      if (!finite_pos(w0[m])) return fail(HOT_EINVAL, "hot_set_traps: weight %d not finite and > 0", m);
  // Eq. 2 in turns per pixel index: a = x p/(lambda f), b = y p/(lambda f), c = z p^2/(2 lambda f^2)
  double *abc = static_cast<double *>(malloc(sizeof(double) * 3 * M));
  float *wh = static_cast<float *>(malloc(sizeof(float) * M));
  if (!abc || !wh) {
    free(abc);
    free(wh);
    return fail(HOT_ENOMEM, "hot_set_traps: out of host memory");
  }
  const double lin = c->pitch / (c->lam * c->focal);
  const double quad = c->pitch * c->pitch / (2.0 * c->lam * c->focal * c->focal);
  for (int m = 0; m < M; m++) {
    abc[3 * m] = xyz_m[3 * m] * lin;
    abc[3 * m + 1] = xyz_m[3 * m + 1] * lin;
    abc[3 * m + 2] = xyz_m[3 * m + 2] * quad;
    wh[m] = w0 ? (float)w0[m] : 1.0f;
  }
  int rc = HOT_OK;
  if (M != c->M) {
    cudaStreamSynchronize(c->st);
    free_traps(c);
    c->M = M;
    rc = build_schedule(c);
    c->M = 0;
    if (rc != HOT_OK) {
      free(abc);
      free(wh);
      return rc;
    }
    rc = dalloc(&c->abc, 3 * (size_t)M);
    if (rc == HOT_OK) rc = dalloc(&c->Xt, (size_t)M * c->W);
    if (rc == HOT_OK) rc = dalloc(&c->Xr, (size_t)M * c->W);
    if (rc == HOT_OK) rc = dalloc(&c->Yt, (size_t)M * c->H);
    if (rc == HOT_OK) rc = dalloc(&c->Yr, (size_t)M * c->H);
    // shifted row tables: rows y0 .. y0 + 15 of copy (4 - y0 % 4) % 4 start 16-byte aligned
    c->ldy4 = (c->H + 18 + 3) & ~3;
    if (rc == HOT_OK) rc = dalloc(&c->Y4t, 4 * (size_t)M * c->ldy4);
    if (rc == HOT_OK) rc = dalloc(&c->Y4r, 4 * (size_t)M * c->ldy4);
    if (rc == HOT_OK && (cudaMemsetAsync(c->Y4t, 0, sizeof(float) * 4 * (size_t)M * c->ldy4, c->st) != cudaSuccess ||
                         cudaMemsetAsync(c->Y4r, 0, sizeof(float) * 4 * (size_t)M * c->ldy4, c->st) != cudaSuccess))
      rc = fail(HOT_ECUDA, "hot_set_traps: clearing the shifted row tables failed");
    if (rc == HOT_OK) rc = dalloc(&c->Xc, (size_t)M * c->W);
    if (rc == HOT_OK) rc = dalloc(&c->Yc, (size_t)M * c->H);
    if (rc == HOT_OK) rc = dalloc(&c->Yc2, 2 * (size_t)M * c->ldy4);
    if (rc == HOT_OK && cudaMemsetAsync(c->Yc2, 0, sizeof(float2) * 2 * (size_t)M * c->ldy4, c->st) != cudaSuccess)
      rc = fail(HOT_ECUDA, "hot_set_traps: clearing the shifted complex row table failed");
    if (rc == HOT_OK) rc = dalloc(&c->w, 2 * (size_t)M);
    if (rc == HOT_OK) rc = dalloc(&c->acc, acc_elems(M));
    if (rc == HOT_OK) rc = dalloc(&c->Vsum, 2 * (size_t)M);
    if (rc == HOT_OK && cudaMemsetAsync(c->acc, 0, sizeof(unsigned long long) * acc_elems(M), c->st) != cudaSuccess)
      rc = fail(HOT_ECUDA, "hot_set_traps: clearing the field accumulators failed");
    if (rc != HOT_OK) {
      free_traps(c);
      free(abc);
      free(wh);
      return rc;
    }
    c->M = M;
  }
  cudaError_t e = cudaMemcpyAsync(c->abc, abc, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->w, wh, sizeof(float) * M, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);  // host buffers are released below
  free(abc);
  free(wh);
  if (e != cudaSuccess) return fail(HOT_ECUDA, "hot_set_traps: %s", cudaGetErrorString(e));
  c->have_fields = false;
  c->u_valid = false;
  return launch_build_tables(c);
}

int hot_set_weights(hot_ctx *c, const double *w) {
  if (!c || !w) return fail(HOT_EINVAL, "hot_set_weights: NULL argument");
  if (!c->M) return fail(HOT_ESTATE, "hot_set_weights: no traps set");
  std::vector<float> wf(c->M);
  for (int m = 0; m < c->M; m++) {
    if (!finite_pos(w[m])) return fail(HOT_EINVAL, "hot_set_weights: weight %d not finite and > 0", m);
    wf[m] = (float)w[m];
  }
  HOT_CUDA(cudaMemcpyAsync(c->w, wf.data(), sizeof(float) * c->M, cudaMemcpyHostToDevice, c->st));
  HOT_CUDA(cudaStreamSynchronize(c->st));
  return HOT_OK;
}

int hot_set_phase(hot_ctx *c, const float *phi, int on_device) {
  if (!c || !phi) return fail(HOT_EINVAL, "hot_set_phase: NULL argument");
  const size_t bytes = sizeof(float) * (size_t)c->W * c->H;
  if (on_device) {
    HOT_CUDA(cudaMemcpyAsync(c->phi, phi, bytes, cudaMemcpyDeviceToDevice, c->st));
  } else {
    HOT_CUDA(cudaMemcpyAsync(c->phi, phi, bytes, cudaMemcpyHostToDevice, c->st));
    HOT_CUDA(cudaStreamSynchronize(c->st));
  }
  c->have_fields = false;
  c->u_valid = false;
  return HOT_OK;
}

int hot_set_precision(hot_ctx *c, int precision) {
  if (!c) return fail(HOT_EINVAL, "hot_set_precision: NULL context");
  if (precision != HOT_PREC_ACCURATE && precision != HOT_PREC_FAST && precision != HOT_PREC_SEPARABLE &&
      precision != HOT_PREC_TENSOR)
    return fail(HOT_EINVAL, "hot_set_precision: unknown mode %d", precision);
  const bool was_sep = separable_kernels(c);
  const bool copies_change = (precision == HOT_PREC_SEPARABLE) != (c->precision == HOT_PREC_SEPARABLE);
  if (was_sep != (precision == HOT_PREC_SEPARABLE || precision == HOT_PREC_TENSOR) || copies_change)
    HOT_CUDA(cudaStreamSynchronize(c->st));
  const bool resched = was_sep != (precision == HOT_PREC_SEPARABLE || precision == HOT_PREC_TENSOR);
  c->precision = precision;
  c->u_valid = false;
  if (resched && c->M) return build_schedule(c);  // the two kernels' occupancies differ
  return HOT_OK;
}

int hot_gsw(hot_ctx *c, int iters, double *eff_out, double *unif_out) {
  if (!c) return fail(HOT_EINVAL, "hot_gsw: NULL context");
  if (iters < 0) return fail(HOT_EINVAL, "hot_gsw: iters = %d < 0", iters);
  if (!c->M) return fail(HOT_ESTATE, "hot_gsw: no traps set");
  if (c->precision == HOT_PREC_TENSOR) {
    if (c->persistent) return fail(HOT_EINVAL, "hot_gsw: the persistent form has no tensor-core variant");
    const int rc = ensure_tc_plan(c);
    if (rc != HOT_OK) return rc;
  }
  if (c->tracing) {
    if (iters > c->trace_cap) {  // the launches' trace slots change: recapture the graphs
      HOT_CUDA(cudaStreamSynchronize(c->st));
      drop_graphs(c);
      dfree(c->trace);
      c->trace_cap = 0;
      const int cap = std::max(iters, 64);
      const int rc = dalloc(&c->trace, 2 * (size_t)cap);
      if (rc != HOT_OK) return rc;
      c->trace_cap = cap;
    }
    c->trace_iters = iters;
  }
  const bool had_u = c->u_valid;
  c->gsw_from_u = c->u_valid && c->once && c->ubuf;
  c->u_valid = false;
  const int rc = (c->use_graphs && !c->profiling && !c->persistent) ? launch_gsw_graph(c, iters) : enqueue_gsw(c, iters);
  c->gsw_from_u = false;
  if (rc != HOT_OK) return rc;
  // the last step of the one-exponential form left u_j of the phases it wrote in ubuf
  c->u_valid = iters > 0 ? c->once && c->ubuf : had_u;
  c->have_fields = true;
  if (eff_out || unif_out) {
    if (c->persistent || c->precision == HOT_PREC_TENSOR) {
      const int rc2 = check_wait_error(c, "hot_gsw");
      if (rc2 != HOT_OK) return rc2;
    }
    float m[2];
    HOT_CUDA(cudaMemcpyAsync(m, c->metrics, sizeof m, cudaMemcpyDeviceToHost, c->st));
    HOT_CUDA(cudaStreamSynchronize(c->st));
    if (eff_out) *eff_out = m[0];
    if (unif_out) *unif_out = m[1];
  }
  return HOT_OK;
}

int hot_phase_out(hot_ctx *c, void *dst, int fmt, int on_device) {
  if (!c || !dst) return fail(HOT_EINVAL, "hot_phase_out: NULL argument");
  if (fmt != HOT_FMT_F32 && fmt != HOT_FMT_U8) return fail(HOT_EINVAL, "hot_phase_out: unknown format %d", fmt);
  const size_t N = (size_t)c->W * c->H;
  if (fmt == HOT_FMT_F32) {
    HOT_CUDA(cudaMemcpyAsync(dst, c->phi, N * sizeof(float),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
  } else {
    unsigned char *g = static_cast<unsigned char *>(dst);
    if (!on_device) {
      if (!c->u8) {
        int rc = dalloc(&c->u8, N);
        if (rc != HOT_OK) return rc;
      }
      g = c->u8;
    }
    const int blocks = (int)(((long long)N + 255) / 256 < 8192 ? ((long long)N + 255) / 256 : 8192);
    int rc;
    {
      Probe p(c, HOT_KERNEL_OTHER);
      hot::quantize_kernel<<<blocks, 256, 0, c->st>>>(c->phi, g, (long long)N);
      rc = check_launch(c, "quantize_kernel");
    }
    if (rc != HOT_OK) return rc;
    if (!on_device) HOT_CUDA(cudaMemcpyAsync(dst, c->u8, N, cudaMemcpyDeviceToHost, c->st));
  }
  if (!on_device) HOT_CUDA(cudaStreamSynchronize(c->st));
  return HOT_OK;
}

int hot_get_fields(hot_ctx *c, double *V, double *w) {
  if (!c) return fail(HOT_EINVAL, "hot_get_fields: NULL context");
  if (!c->M) return fail(HOT_ESTATE, "hot_get_fields: no traps set");
  if (V && !c->have_fields) return fail(HOT_ESTATE, "hot_get_fields: no forward evaluation since the last change");
  const int rc = check_wait_error(c, "hot_get_fields");
  if (rc != HOT_OK) return rc;
  std::vector<long long> vs(V ? 2 * c->M : 0);
  std::vector<float> wf(w ? c->M : 0);
  if (V) HOT_CUDA(cudaMemcpyAsync(vs.data(), c->Vsum, sizeof(long long) * 2 * c->M, cudaMemcpyDeviceToHost, c->st));
  if (w) HOT_CUDA(cudaMemcpyAsync(wf.data(), c->w, sizeof(float) * c->M, cudaMemcpyDeviceToHost, c->st));
  HOT_CUDA(cudaStreamSynchronize(c->st));
  const double inv = 1.0 / (n_total(c) * ldexp(1.0, c->fx_shift));
  for (int m = 0; V && m < c->M; m++) {  // fixed-point sums -> V_m
    V[2 * m] = (double)vs[m] * inv;
    V[2 * m + 1] = (double)vs[c->M + m] * inv;
  }
  for (int m = 0; w && m < c->M; m++) w[m] = wf[m];
  return HOT_OK;
}

int hot_field(hot_ctx *c, const float *phi, float *V) {
  if (!c || !phi || !V) return fail(HOT_EINVAL, "hot_field: NULL argument");
  if (!c->M) return fail(HOT_ESTATE, "hot_field: no traps set");
  int rc = launch_mode<false, true>(c, false, 0, phi);
  if (rc == HOT_OK) rc = launch_finalize(c, false, 0);  // w stays in w[0]; accumulators cleared
  if (rc != HOT_OK) return rc;
  const double inv = 1.0 / (n_total(c) * ldexp(1.0, c->fx_shift));
  hot::sums_to_fields_kernel<<<(c->M + 255) / 256, 256, 0, c->st>>>(c->M, c->Vsum, inv, reinterpret_cast<float2 *>(V));
  rc = check_launch(c, "sums_to_fields_kernel");
  if (rc == HOT_OK) c->have_fields = true;
  return rc;
}

int hot_superposition(hot_ctx *c, const double *coef) {
  if (!c || !coef) return fail(HOT_EINVAL, "hot_superposition: NULL argument");
  if (!c->M) return fail(HOT_ESTATE, "hot_superposition: no traps set");
  std::vector<float> cf(2 * (size_t)c->M);
  for (int i = 0; i < 2 * c->M; i++) {
    if (!std::isfinite(coef[i])) return fail(HOT_EINVAL, "hot_superposition: coefficient %d not finite", i / 2);
    cf[i] = (float)coef[i];
  }
  float2 *d = nullptr;
  int rc = dalloc(&d, c->M);
  if (rc != HOT_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(d, cf.data(), sizeof(float) * cf.size(), cudaMemcpyHostToDevice, c->st);
  if (e != cudaSuccess) rc = fail(HOT_ECUDA, "hot_superposition: %s", cudaGetErrorString(e));
  if (rc == HOT_OK)
    rc = launch_mode<true, false>(c, false, 0, nullptr, d);
  if (rc == HOT_OK) {
    e = cudaStreamSynchronize(c->st);  // the coefficients are freed below
    if (e != cudaSuccess) rc = fail(HOT_ECUDA, "hot_superposition: %s", cudaGetErrorString(e));
  }
  dfree(d);
  c->have_fields = false;
  c->u_valid = false;
  return rc;
}

int hot_field_adjoint(hot_ctx *c, const float *phi, const float *G, float *grad) {
  if (!c || !phi || !G || !grad) return fail(HOT_EINVAL, "hot_field_adjoint: NULL argument");
  if (!c->M) return fail(HOT_ESTATE, "hot_field_adjoint: no traps set");
  const float2 *g = reinterpret_cast<const float2 *>(G);
  return launch_mode<true, false, true>(c, false, 0, phi, g, grad);
}

int hot_intensity_loss(hot_ctx *c, const float *phi, double beta, float *loss, float *grad) {
  if (!c || !phi || !loss) return fail(HOT_EINVAL, "hot_intensity_loss: NULL argument");
  if (!c->M) return fail(HOT_ESTATE, "hot_intensity_loss: no traps set");
  if (!std::isfinite(beta)) return fail(HOT_EINVAL, "hot_intensity_loss: beta not finite");
  if (!c->G) {
    const int rc = dalloc(&c->G, c->M);
    if (rc != HOT_OK) return rc;
  }
  int rc = launch_mode<false, true>(c, false, 0, phi);  // sums of V = F(phi) in accumulator 0
  if (rc != HOT_OK) return rc;
  hot::LossArgs a = {};
  a.M = c->M;
  a.copies = acc_copies(c);
  a.acc = c->acc;
  a.acc_all = c->acc;
  a.Vsum = c->Vsum;
  a.metrics = c->metrics;
  a.inv_fx_n = 1.0 / (n_total(c) * ldexp(1.0, c->fx_shift));
  a.beta = beta;
  a.G = c->G;
  a.loss = loss;
  {
    Probe p(c, HOT_KERNEL_FINISH);
    hot::intensity_loss_kernel<<<1, hot::kLossThreads, 0, c->st>>>(a);
  }
  rc = check_launch(c, "intensity_loss_kernel");
  if (rc != HOT_OK) return rc;
  c->have_fields = true;
  if (!grad) return HOT_OK;
  return launch_mode<true, false, true>(c, false, 0, phi, c->G, grad);
}

int hot_set_band(hot_ctx *c, int total_height, int y0) {
  if (!c) return fail(HOT_EINVAL, "hot_set_band: NULL context");
  if (total_height < c->H || y0 < 0 || y0 > total_height - c->H || (long long)c->W * total_height >= (1LL << 31))
    return fail(HOT_EINVAL, "hot_set_band: rows %d .. %d not inside a hologram of %d rows", y0, y0 + c->H - 1,
                total_height);
  HOT_CUDA(cudaStreamSynchronize(c->st));
  drop_graphs(c);
  c->H_total = total_height;
  c->y_off = y0;
  c->fx_shift = fixed_point_shift((long long)c->W * total_height);
  c->have_fields = false;
  c->u_valid = false;
  c->shard_k = -1;
  return c->M ? launch_build_tables(c) : HOT_OK;
}

int hot_sharded_begin(hot_ctx *c) {
  if (!c) return fail(HOT_EINVAL, "hot_sharded_begin: NULL context");
  if (!c->M) return fail(HOT_ESTATE, "hot_sharded_begin: no traps set");
  c->shard_k = -1;
  c->have_fields = false;
  c->u_valid = false;
  int rc = HOT_OK;
  if (c->precision == HOT_PREC_TENSOR) {
    rc = ensure_tc_plan(c);
    if (rc == HOT_OK) rc = launch_tc(c, false, 0);
  } else {
    rc = launch_step(c, false, true, false, 0);
  }
  if (rc == HOT_OK) c->shard_k = 0;
  return rc;
}

int hot_sharded_step(hot_ctx *c, int k) {
  if (!c) return fail(HOT_EINVAL, "hot_sharded_step: NULL context");
  if (c->shard_k < 0 || k != c->shard_k + 1)
    return fail(HOT_ESTATE, "hot_sharded_step: launch %d does not follow launch %d", k, c->shard_k);
  const int rc = c->precision == HOT_PREC_TENSOR ? launch_tc(c, false, k) : launch_step(c, true, true, false, k);
  if (rc == HOT_OK) c->shard_k = k;
  return rc;
}

int hot_sharded_sums(hot_ctx *c, int k, void **sums_dev, int *count) {
  if (!c || !sums_dev || !count) return fail(HOT_EINVAL, "hot_sharded_sums: NULL argument");
  if (c->shard_k < 0 || k != c->shard_k)
    return fail(HOT_ESTATE, "hot_sharded_sums: launch %d is not the last one (%d)", k, c->shard_k);
  const size_t n = 2 * (size_t)c->M * acc_copies(c);
  *sums_dev = c->acc + n * (k % 3);
  *count = (int)n;
  return HOT_OK;
}

int hot_sharded_end(hot_ctx *c, int iters, double *eff_out, double *unif_out) {
  if (!c) return fail(HOT_EINVAL, "hot_sharded_end: NULL context");
  if (c->shard_k < 0 || iters != c->shard_k)
    return fail(HOT_ESTATE, "hot_sharded_end: iters = %d, last launch %d", iters, c->shard_k);
  const int rc = launch_finalize(c, false, iters);
  c->shard_k = -1;
  if (rc != HOT_OK) return rc;
  c->have_fields = true;
  if (eff_out || unif_out) {
    float m[2];
    HOT_CUDA(cudaMemcpyAsync(m, c->metrics, sizeof m, cudaMemcpyDeviceToHost, c->st));
    HOT_CUDA(cudaStreamSynchronize(c->st));
    if (eff_out) *eff_out = m[0];
    if (unif_out) *unif_out = m[1];
  }
  return HOT_OK;
}

int hot_get_metrics(hot_ctx *c, double *eff_out, double *unif_out) {
  if (!c) return fail(HOT_EINVAL, "hot_get_metrics: NULL context");
  if (!c->M || !c->have_fields) return fail(HOT_ESTATE, "hot_get_metrics: no forward evaluation since the last change");
  const int rc = check_wait_error(c, "hot_get_metrics");
  if (rc != HOT_OK) return rc;
  float m[2];
  HOT_CUDA(cudaMemcpyAsync(m, c->metrics, sizeof m, cudaMemcpyDeviceToHost, c->st));
  HOT_CUDA(cudaStreamSynchronize(c->st));
  if (eff_out) *eff_out = m[0];
  if (unif_out) *unif_out = m[1];
  return HOT_OK;
}

int hot_sync(hot_ctx *c) {
  if (!c) return fail(HOT_EINVAL, "hot_sync: NULL context");
  HOT_CUDA(cudaStreamSynchronize(c->st));
  return check_wait_error(c, "hot_sync");
}

int hot_set_trace(hot_ctx *c, int enable) {
  if (!c) return fail(HOT_EINVAL, "hot_set_trace: NULL context");
  if ((enable != 0) != c->tracing) {
    HOT_CUDA(cudaStreamSynchronize(c->st));
    drop_graphs(c);  // the captured launches carry (or not) trace slots
  }
  c->tracing = enable != 0;
  c->trace_iters = -1;
  return HOT_OK;
}

int hot_get_trace(hot_ctx *c, double *eff, double *unif, int n) {
  if (!c || !eff || !unif) return fail(HOT_EINVAL, "hot_get_trace: NULL argument");
  if (!c->tracing || c->trace_iters < 0 || !c->have_fields)
    return fail(HOT_ESTATE, "hot_get_trace: no traced hot_gsw since tracing was enabled");
  const int K = c->trace_iters;
  if (n != K + 1) return fail(HOT_EINVAL, "hot_get_trace: n = %d, the last call has %d values", n, K + 1);
  const int rc = check_wait_error(c, "hot_get_trace");
  if (rc != HOT_OK) return rc;
  std::vector<float> t(2 * (size_t)K + 2);
  if (K) HOT_CUDA(cudaMemcpyAsync(t.data(), c->trace, sizeof(float) * 2 * K, cudaMemcpyDeviceToHost, c->st));
  HOT_CUDA(cudaMemcpyAsync(t.data() + 2 * K, c->metrics, sizeof(float) * 2, cudaMemcpyDeviceToHost, c->st));
  HOT_CUDA(cudaStreamSynchronize(c->st));
  for (int k = 0; k <= K; k++) {
    eff[k] = t[2 * k];
    unif[k] = t[2 * k + 1];
  }
  return HOT_OK;
}

int hot_get_state(hot_ctx *c, float *phi, float *w) {
  if (!c || !phi || !w) return fail(HOT_EINVAL, "hot_get_state: NULL argument");
  if (!c->M) return fail(HOT_ESTATE, "hot_get_state: no traps set");
  const int rc = check_wait_error(c, "hot_get_state");
  if (rc != HOT_OK) return rc;
  HOT_CUDA(cudaMemcpyAsync(phi, c->phi, sizeof(float) * (size_t)c->W * c->H, cudaMemcpyDeviceToHost, c->st));
  HOT_CUDA(cudaMemcpyAsync(w, c->w, sizeof(float) * c->M, cudaMemcpyDeviceToHost, c->st));
  HOT_CUDA(cudaStreamSynchronize(c->st));
  return HOT_OK;
}

int hot_set_state(hot_ctx *c, const float *phi, const float *w) {
  if (!c || !phi || !w) return fail(HOT_EINVAL, "hot_set_state: NULL argument");
  if (!c->M) return fail(HOT_ESTATE, "hot_set_state: no traps set");
  for (int m = 0; m < c->M; m++)
    if (!(std::isfinite(w[m]) && w[m] > 0.f)) return fail(HOT_EINVAL, "hot_set_state: weight %d not finite and > 0", m);
  HOT_CUDA(cudaMemcpyAsync(c->phi, phi, sizeof(float) * (size_t)c->W * c->H, cudaMemcpyHostToDevice, c->st));
  HOT_CUDA(cudaMemcpyAsync(c->w, w, sizeof(float) * c->M, cudaMemcpyHostToDevice, c->st));
  HOT_CUDA(cudaStreamSynchronize(c->st));
  c->have_fields = false;
  c->u_valid = false;
  return HOT_OK;
}

int hot_get_phasors(hot_ctx *c, float *u) {
  if (!c || !u) return fail(HOT_EINVAL, "hot_get_phasors: NULL argument");
  if (!c->M) return fail(HOT_ESTATE, "hot_get_phasors: no traps set");
  if (!c->u_valid)
    return fail(HOT_ESTATE, "hot_get_phasors: no unit phasors of the current phases (a one-exponential hot_gsw leaves them)");
  const int rc = check_wait_error(c, "hot_get_phasors");
  if (rc != HOT_OK) return rc;
  HOT_CUDA(cudaMemcpyAsync(u, c->ubuf, sizeof(float2) * (size_t)c->W * c->H, cudaMemcpyDeviceToHost, c->st));
  HOT_CUDA(cudaStreamSynchronize(c->st));
  return HOT_OK;
}

int hot_set_phasors(hot_ctx *c, const float *u) {
  if (!c || !u) return fail(HOT_EINVAL, "hot_set_phasors: NULL argument");
  if (!c->M) return fail(HOT_ESTATE, "hot_set_phasors: no traps set");
  if (!c->once || !c->ubuf) return fail(HOT_ESTATE, "hot_set_phasors: the one-exponential step is not in effect");
  const size_t n = 2 * (size_t)c->W * c->H;
  for (size_t i = 0; i < n; i++)
    if (!std::isfinite(u[i]) || std::fabs(u[i]) > 2.f)
      return fail(HOT_EINVAL, "hot_set_phasors: value %zu is not a unit phasor component", i);
  HOT_CUDA(cudaMemcpyAsync(c->ubuf, u, sizeof(float) * n, cudaMemcpyHostToDevice, c->st));
  HOT_CUDA(cudaStreamSynchronize(c->st));
  c->u_valid = true;
  return HOT_OK;
}

int hot_use_persistent(hot_ctx *c, int enable) {
  if (!c) return fail(HOT_EINVAL, "hot_use_persistent: NULL context");
  c->persistent = enable != 0;
  return HOT_OK;
}

int hot_set_wait_limit(hot_ctx *c, double seconds) {
  if (!c) return fail(HOT_EINVAL, "hot_set_wait_limit: NULL context");
  if (!(seconds >= 0.0) || seconds > 60.0) return fail(HOT_EINVAL, "hot_set_wait_limit: %g s not in [0, 60]", seconds);
  c->wait_limit_s = seconds;
  return HOT_OK;
}

long long hot_kernel_launches(const hot_ctx *c) { return c ? c->launches : 0; }

int hot_use_graphs(hot_ctx *c, int enable) {
  if (!c) return fail(HOT_EINVAL, "hot_use_graphs: NULL context");
  c->use_graphs = enable != 0;
  return HOT_OK;
}

int hot_profile(hot_ctx *c, int enable) {
  if (!c) return fail(HOT_EINVAL, "hot_profile: NULL context");
  if (!enable && c->profiling) {
    HOT_CUDA(cudaStreamSynchronize(c->st));
    clear_records(c);
  }
  c->profiling = enable != 0;
  return HOT_OK;
}

int hot_profile_read(hot_ctx *c, double *ms, long long *launches) {
  if (!c) return fail(HOT_EINVAL, "hot_profile_read: NULL context");
  HOT_CUDA(cudaStreamSynchronize(c->st));
  double t[HOT_KERNEL_KINDS] = {0, 0, 0, 0};
  long long n[HOT_KERNEL_KINDS] = {0, 0, 0, 0};
  for (auto &r : c->recs) {
    float x = 0.f;
    cudaError_t e = cudaEventElapsedTime(&x, r.a, r.b);
    if (e != cudaSuccess) {
      clear_records(c);
      return fail(HOT_ECUDA, "hot_profile_read: %s", cudaGetErrorString(e));
    }
    t[r.kind] += x;
    n[r.kind] += 1;
  }
  clear_records(c);
  for (int k = 0; k < HOT_KERNEL_KINDS; k++) {
    if (ms) ms[k] = t[k];
    if (launches) launches[k] = n[k];
  }
  return HOT_OK;
}

}  // extern "C"


// ---------------------------------------------------------------------------------------------
// Batches of holograms (hot_batch_*).
struct hot_batch {
  int count = 0, precision = HOT_PREC_ACCURATE, dev = 0;
  std::vector<hot_ctx *> ctx;
  cudaStream_t st = nullptr, cap = nullptr;
  int sms = 0, per_sm_max = 1;
  // tiling (hot_batch_set_tiling) and group threshold in pixel-trap pairs per iteration
  int rows = hot::kRowsMax, bps = 0, chunk = hot::kChunk;
  double group_pairs = 67108864.0;
  struct Group {
    std::vector<int> members;         // context indices (<= kBatchMax); SubTile::pad indexes this list
    int grid = 0, n_sub = 0;
    hot::SubTile *sub = nullptr;
    int *first = nullptr;
    std::vector<int> owner;                  // block that writes each hologram's weights
    std::vector<hot::StepArgs> holo[6];      // parameters for launch k (k % 6; k = 0 uses set 0)
    hot::FinalizeArgs *fin[6] = {};          // finalize descriptors for iters % 6
  };
  std::vector<Group> groups;
  unsigned long long *stamps = nullptr;  // [count + 1]: completion of hologram h; [count]: start
  bool ran = false;
  // HOT_PREC_TENSOR: each member runs its own hot_gsw launch sequence; the members are dealt out
  // to up to kTensorChains streams (largest work first, each to the least loaded chain) whose
  // launches overlap, forked from and joined to the batch's stream inside its graph
  std::vector<std::vector<int>> chains;
  std::vector<cudaStream_t> chain_st;
  std::vector<cudaEvent_t> chain_ev;  // [0]: fork; [1 + i]: end of chain i

  struct Graph {
    int iters;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
};

namespace {

int batch_mode(const hot_batch *b) {
  return b->precision == HOT_PREC_SEPARABLE ? hot::kModeSeparable
                                            : b->precision == HOT_PREC_FAST ? hot::kModeFast : hot::kModeAccurate;
}

// Dynamic shared memory of the batch kernels: the separable one stages `chunk` complex traps.
int batch_smem(const hot_batch *b) {
  return b->precision == HOT_PREC_SEPARABLE ? hot::sep_smem_bytes(b->chunk) : hot::step_smem_bytes(0, true);
}

template <int MODE>
int batch_set_smem() {
  const int bytes = MODE == hot::kModeSeparable ? hot::sep_smem_bytes(hot::kChunk) : hot::step_smem_bytes(0, true);
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_batch_kernel<MODE, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_batch_kernel<MODE, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return HOT_OK;
}

// Resident blocks per SM of the batch's fused kernel at its current staging chunk.
int batch_occupancy(hot_batch *b) {
  int per_sm = 0;
  const int smem = batch_smem(b);
  cudaError_t e;
  switch (batch_mode(b)) {
    case hot::kModeSeparable:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hot::gsw_batch_kernel<hot::kModeSeparable, true, true>,
                                                        hot::kThreads, smem);
      break;
    case hot::kModeFast:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hot::gsw_batch_kernel<hot::kModeFast, true, true>,
                                                        hot::kThreads, smem);
      break;
    default:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hot::gsw_batch_kernel<hot::kModeAccurate, true, true>,
                                                        hot::kThreads, smem);
  }
  if (e != cudaSuccess) return fail(HOT_ECUDA, "batch occupancy query: %s", cudaGetErrorString(e));
  b->per_sm_max = per_sm < 1 ? 1 : per_sm;
  return HOT_OK;
}

void batch_drop_graphs(hot_batch *b) {
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
}

void group_free(hot_batch::Group &g) {
  dfree(g.sub);
  dfree(g.first);
  for (auto &p : g.fin) dfree(p);
}

void batch_free(hot_batch *b) {
  batch_drop_graphs(b);
  for (auto &g : b->groups) group_free(g);
  b->groups.clear();
  dfree(b->stamps);
  if (b->cap) cudaStreamDestroy(b->cap);
  b->cap = nullptr;
  for (cudaStream_t s : b->chain_st) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->chain_ev) cudaEventDestroy(e);
  b->chain_st.clear();
  b->chain_ev.clear();
}

// Step-kernel parameters of context c for launch k of a sequence (buffers rotate as in hot_gsw).
hot::StepArgs step_args(const hot_ctx *c, int k, int chunk) {
  hot::StepArgs a = {};
  const bool fast = c->precision == HOT_PREC_FAST;
  const size_t M2 = 2 * (size_t)c->M * acc_copies(c);
  a.W = c->W;
  a.H = c->H;
  a.M = c->M;
  a.chunk = chunk;
  a.copies = acc_copies(c);
  a.X = fast ? c->Xr : c->Xt;
  a.Y = fast ? c->Yr : c->Yt;
  a.Y4 = fast ? c->Y4r : c->Y4t;
  a.ldy4 = c->ldy4;
  a.Xc = c->Xc;
  a.Yc = c->Yc2;
  a.phi = c->phi;
  a.acc_in = c->acc + M2 * ((k + 2) % 3);
  a.acc_out = c->acc + M2 * (k % 3);
  a.acc_clear = c->acc + M2 * ((k + 1) % 3);
  a.w_in = c->w + (size_t)c->M * ((k + 1) & 1);
  a.w_out = c->w + (size_t)c->M * (k & 1);
  a.fx_scale = ldexpf(1.0f, c->fx_shift);
  a.inv_fx_n = (float)(1.0 / (n_total(c) * ldexp(1.0, c->fx_shift)));
  a.angle_units = fast ? 1.0f : 0.15915494309189535f;
  a.angle_eta = fast ? hot::kFastEta : 0.0f;
  a.inv_n = (float)(1.0 / (n_total(c)));
  return a;
}

double pairs_of(const hot_ctx *c) { return n_total(c) * (double)c->M; }

// One group's work schedule: the row segments of its holograms in order, each weighted by its
// trap count, dealt out to one wave of G blocks in equal shares (a segment goes to the block
// that holds the midpoint of its weight interval); each block's run of rows in a strip is cut
// into equal sub-tiles of <= rows rows.
int build_group(hot_batch *b, hot_batch::Group &g) {
  const int count = (int)g.members.size();
  const int per_sm = b->bps > 0 ? std::min(b->bps, b->per_sm_max) : b->per_sm_max;
  long double T = 0;
  long long segments = 0;
  for (int h : g.members) {
    const hot_ctx *c = b->ctx[h];
    const long long seg = (long long)((c->W + hot::kTileW - 1) / hot::kTileW) * c->H;
    segments += seg;
    T += (long double)seg * c->M;
  }
  const int G = (int)std::min<long long>((long long)b->sms * per_sm, segments);
  std::vector<hot::SubTile> sub;
  std::vector<int> first(G + 1, 0), owner(count, -1);
  long double w0 = 0;
  int cur_b = 0;
  for (int i = 0; i < count; i++) {
    const hot_ctx *c = b->ctx[g.members[i]];
    const int strips = (c->W + hot::kTileW - 1) / hot::kTileW;
    for (int s = 0; s < strips; s++) {
      auto block_of = [&](int row) {
        const long double mid = w0 + ((long double)row + 0.5L) * c->M;
        const int bb = (int)(mid * G / T);
        return bb < 0 ? 0 : (bb >= G ? G - 1 : bb);
      };
      int r = 0;
      while (r < c->H) {  // the run of rows of this strip that goes to block bb, cut evenly
        const int bb = block_of(r);
        int r1 = r + 1;
        while (r1 < c->H && block_of(r1) == bb) r1++;
        while (cur_b < bb) first[++cur_b] = (int)sub.size();
        if (owner[i] < 0) owner[i] = bb;
        const int L = r1 - r, nsub = (L + b->rows - 1) / b->rows;
        for (int q = 0; q < nsub; q++) {
          const int q0 = r + (int)((long long)L * q / nsub), q1 = r + (int)((long long)L * (q + 1) / nsub);
          sub.push_back({s * hot::kTileW, q0, q1 - q0, i});
        }
        r = r1;
      }
      w0 += (long double)c->H * c->M;
    }
  }
  while (cur_b < G) first[++cur_b] = (int)sub.size();
  g.grid = G;
  g.n_sub = (int)sub.size();
  g.owner = owner;
  for (int k = 0; k < 6; k++) {
    g.holo[k].resize(count);
    for (int i = 0; i < count; i++) g.holo[k][i] = step_args(b->ctx[g.members[i]], k == 0 ? 6 : k, b->chunk);
  }
  int rc = dalloc(&g.sub, sub.size());
  if (rc == HOT_OK) rc = dalloc(&g.first, first.size());
  for (int r6 = 0; rc == HOT_OK && r6 < 6; r6++) {  // finalize after `iters` iterations, iters % 6 == r6
    rc = dalloc(&g.fin[r6], (size_t)count);
    std::vector<hot::FinalizeArgs> fs(count);
    for (int i = 0; i < count; i++) {
      const hot_ctx *c = b->ctx[g.members[i]];
      hot::FinalizeArgs &f = fs[i];
      f.M = c->M;
      f.copies = acc_copies(c);
      f.acc = c->acc + 2 * (size_t)c->M * acc_copies(c) * (r6 % 3);  // the last launch accumulated into acc[iters % 3]
      f.acc_all = c->acc;
      f.w_src = c->w + (size_t)c->M * (r6 & 1);       // and left the weights in w[iters & 1]
      f.w_dst = c->w;
      f.Vsum = c->Vsum;
      f.metrics = c->metrics;
      f.inv_fx_n = (float)(1.0 / (n_total(c) * ldexp(1.0, c->fx_shift)));
      f.done = b->stamps + g.members[i];
    }
    if (rc == HOT_OK && cudaMemcpy(g.fin[r6], fs.data(), sizeof(hot::FinalizeArgs) * count, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = fail(HOT_ECUDA, "batch schedule: copy of descriptors failed");
  }
  if (rc == HOT_OK) {
    cudaError_t e = cudaMemcpy(g.sub, sub.data(), sizeof(hot::SubTile) * sub.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g.first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = fail(HOT_ECUDA, "batch schedule: %s", cudaGetErrorString(e));
  }
  return rc;
}

// Orders the holograms by pairs per iteration (smallest first, stable), cuts them into
// groups of >= group_pairs (a short last group joins the one before) and builds each group.
int batch_schedule(hot_batch *b) {
  HOT_CUDA(cudaStreamSynchronize(b->st));
  batch_drop_graphs(b);
  const int rc0 = batch_occupancy(b);
  if (rc0 != HOT_OK) return rc0;
  for (auto &g : b->groups) group_free(g);
  b->groups.clear();
  b->ran = false;
  std::vector<int> order(b->count);
  for (int h = 0; h < b->count; h++) order[h] = h;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return pairs_of(b->ctx[x]) < pairs_of(b->ctx[y]); });
  std::vector<std::vector<int>> parts;
  double sum = 0;
  for (int h : order) {
    if (parts.empty() || sum >= b->group_pairs || (int)parts.back().size() == hot::kBatchMax) {
      parts.emplace_back();
      sum = 0;
    }
    parts.back().push_back(h);
    sum += pairs_of(b->ctx[h]);
  }
  if (parts.size() > 1 && sum < b->group_pairs && parts.back().size() + parts[parts.size() - 2].size() <= hot::kBatchMax) {
    auto last = parts.back();
    parts.pop_back();
    parts.back().insert(parts.back().end(), last.begin(), last.end());
  }
  b->groups.resize(parts.size());
  for (size_t i = 0; i < parts.size(); i++) {
    b->groups[i].members = parts[i];
    const int rc = build_group(b, b->groups[i]);
    if (rc != HOT_OK) {
      for (auto &g : b->groups) group_free(g);
      b->groups.clear();
      return rc;
    }
  }
  return HOT_OK;
}

template <int MODE, bool BACK>
int batch_launch(hot_batch *b, const hot_batch::Group &g, int k, bool pdl) {
  hot::BatchArgs a = {};
  const int count = (int)g.members.size();
  for (int i = 0; i < count; i++) {
    a.holo[i] = g.holo[k % 6][i];
    a.owner[i] = g.owner[i];
  }
  a.sub = g.sub;
  a.first = g.first;
  a.count = count;
  hot_ctx tmp;  // launch() needs a context only for the stream
  tmp.st = b->st;
  launch(&tmp, hot::gsw_batch_kernel<MODE, BACK, true>, g.grid, hot::kThreads, batch_smem(b), pdl, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(HOT_ECUDA, "launch of gsw_batch_kernel: %s", cudaGetErrorString(e));
  return HOT_OK;
}

// A start stamp, then the groups in order: forward field of the starting phases (k = 0),
// iterations 1..iters, and the per-hologram finalize with its completion stamp.
template <bool BACK>
int batch_launch_mode(hot_batch *b, const hot_batch::Group &g, int k, bool pdl) {
  switch (batch_mode(b)) {
    case hot::kModeSeparable: return batch_launch<hot::kModeSeparable, BACK>(b, g, k, pdl);
    case hot::kModeFast: return batch_launch<hot::kModeFast, BACK>(b, g, k, pdl);
    default: return batch_launch<hot::kModeAccurate, BACK>(b, g, k, pdl);
  }
}

constexpr int kTensorChains = 8;

// Tensor-mode batch set-up: every member's tensor-core operands, and its chain (largest work
// N M first, each to the chain with the least work so far).
int batch_setup_tensor(hot_batch *b) {
  for (hot_ctx *c : b->ctx) {
    const int rc = ensure_tc_plan(c);
    if (rc != HOT_OK) return rc;
    HOT_CUDA(cudaStreamSynchronize(c->st));
  }
  const int n = std::min(b->count, kTensorChains);
  std::vector<int> order(b->count);
  for (int h = 0; h < b->count; h++) order[h] = h;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return pairs_of(b->ctx[x]) > pairs_of(b->ctx[y]); });
  std::vector<double> load(n, 0.0);
  b->chains.assign(n, {});
  for (int h : order) {
    const int i = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->chains[i].push_back(h);
    load[i] += pairs_of(b->ctx[h]);
  }
  b->chain_st.assign(n, nullptr);
  b->chain_ev.assign(n + 1, nullptr);
  for (int i = 0; i < n; i++) HOT_CUDA(cudaStreamCreateWithFlags(&b->chain_st[i], cudaStreamNonBlocking));
  for (int i = 0; i <= n; i++) HOT_CUDA(cudaEventCreateWithFlags(&b->chain_ev[i], cudaEventDisableTiming));
  return HOT_OK;
}

// Tensor-mode batch: a start stamp, then every chain on its own stream (forked from the batch's
// stream by an event), each member's hot_gsw sequence followed by its completion stamp, and the
// chains joined back.  Each member computes exactly what hot_gsw(iters) computes for it.
int batch_enqueue_tensor(hot_batch *b, int iters) {
  hot::stamp_kernel<<<1, 1, 0, b->st>>>(b->stamps + b->count);
  HOT_CUDA(cudaGetLastError());
  HOT_CUDA(cudaEventRecord(b->chain_ev[0], b->st));
  for (size_t i = 0; i < b->chains.size(); i++) {
    cudaStream_t s = b->chain_st[i];
    HOT_CUDA(cudaStreamWaitEvent(s, b->chain_ev[0], 0));
    for (int h : b->chains[i]) {
      hot_ctx *c = b->ctx[h];
      cudaStream_t own = c->st;
      c->st = s;
      const int rc = enqueue_gsw(c, iters);
      c->st = own;
      if (rc != HOT_OK) return rc;
      hot::stamp_kernel<<<1, 1, 0, s>>>(b->stamps + h);
      HOT_CUDA(cudaGetLastError());
    }
    HOT_CUDA(cudaEventRecord(b->chain_ev[1 + i], s));
    HOT_CUDA(cudaStreamWaitEvent(b->st, b->chain_ev[1 + i], 0));
  }
  return HOT_OK;
}

int batch_enqueue(hot_batch *b, int iters) {
  if (b->precision == HOT_PREC_TENSOR) return batch_enqueue_tensor(b, iters);
  hot::stamp_kernel<<<1, 1, 0, b->st>>>(b->stamps + b->count);
  cudaError_t e0 = cudaGetLastError();
  if (e0 != cudaSuccess) return fail(HOT_ECUDA, "launch of stamp_kernel: %s", cudaGetErrorString(e0));
  for (size_t gi = 0; gi < b->groups.size(); gi++) {
    const hot_batch::Group &g = b->groups[gi];
    int rc = batch_launch_mode<false>(b, g, 0, true);
    for (int k = 1; k <= iters && rc == HOT_OK; k++) rc = batch_launch_mode<true>(b, g, k, true);
    if (rc != HOT_OK) return rc;
    hot_ctx tmp;
    tmp.st = b->st;
    launch(&tmp, hot::gsw_finalize_batch_kernel, (int)g.members.size(), hot::kFinalizeThreads, 0, true,
           (const hot::FinalizeArgs *)g.fin[iters % 6]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HOT_ECUDA, "launch of gsw_finalize_batch_kernel: %s", cudaGetErrorString(e));
  }
  return HOT_OK;
}

int check_tiling(const char *who, int rows, int bps, int chunk) {
  if (rows < 0 || rows > hot::kRowsMax) return fail(HOT_EINVAL, "%s: rows = %d not in [1, %d] (0: default)", who, rows, hot::kRowsMax);
  if (bps < 0 || bps > 32) return fail(HOT_EINVAL, "%s: blocks_per_sm = %d not in [1, 32] (0: default)", who, bps);
  if (chunk < 0 || chunk > hot::kChunk) return fail(HOT_EINVAL, "%s: chunk = %d not in [1, %d] (0: default)", who, chunk, hot::kChunk);
  return HOT_OK;
}

struct Tiling {
  int rows, bps, chunk, merge;
  bool operator==(const Tiling &o) const {
    return rows == o.rows && bps == o.bps && chunk == o.chunk && merge == o.merge;
  }
};

// The kernels are launch-bounded to at most 4 resident blocks per SM; a candidate above what
// the current staging chunk leaves room for is clamped to it by the schedule.
constexpr int kMaxBlocksPerSm = 4;

// Coordinate search: each parameter in turn takes the fastest of its candidates with the
// others fixed; a candidate replaces the incumbent only if it is more than 1 % faster; at
// most two passes.  apply(t) installs a tiling, time(&us) measures it.  Leaves `best` applied.
// With merge, the blocks-per-SM candidates include max_bps blocks merged four and two to a
// launched block (Tiling::merge: schedule blocks per launched block).
template <typename Apply, typename Time>
int tune_tiling(int max_bps, Tiling &best, double &best_us, Apply apply, Time time, bool merge = false) {
  static const int rows_c[] = {14, 12, 10, 8, 6, 4, 2};
  static const int chunk_c[] = {128, 96, 64, 32};
  int rc = apply(best);
  if (rc == HOT_OK) rc = time(&best_us);
  for (int pass = 0; rc == HOT_OK && pass < 2; pass++) {
    bool changed = false;
    for (int dim = 0; rc == HOT_OK && dim < 3; dim++) {
      std::vector<int> cand;  // blocks per SM; -4 and -2: max_bps blocks merged 4 or 2 to a block
      if (dim == 0) cand.assign(std::begin(rows_c), std::end(rows_c));
      if (dim == 1) {
        if (merge) {
          cand.push_back(-4);
          cand.push_back(-2);
        }
        for (int v = max_bps; v >= 1; v--) cand.push_back(v);
      }
      if (dim == 2) cand.assign(std::begin(chunk_c), std::end(chunk_c));
      for (int v : cand) {
        Tiling t = best;
        if (dim == 1) {
          t.bps = v < 0 ? max_bps : v;
          t.merge = v < 0 ? -v : 1;
        } else {
          (dim == 0 ? t.rows : t.chunk) = v;
        }
        if (t == best) continue;
        double us = 0;
        rc = apply(t);
        if (rc == HOT_OK) rc = time(&us);
        if (rc != HOT_OK) break;
        if (us < 0.99 * best_us) {
          best = t;
          best_us = us;
          changed = true;
        }
      }
    }
    if (!changed) break;
  }
  const int rc2 = apply(best);
  return rc != HOT_OK ? rc : rc2;
}

// Device copies of phases and weights that an autotuner restores before every timed run.
struct Saved {
  float *phi = nullptr, *w = nullptr;
  ~Saved() {
    dfree(phi);
    dfree(w);
  }
};

int save_state(hot_ctx *c, Saved &s, cudaStream_t st) {
  const size_t N = (size_t)c->W * c->H;
  int rc = dalloc(&s.phi, N);
  if (rc == HOT_OK) rc = dalloc(&s.w, (size_t)c->M);
  if (rc != HOT_OK) return rc;
  HOT_CUDA(cudaMemcpyAsync(s.phi, c->phi, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
  HOT_CUDA(cudaMemcpyAsync(s.w, c->w, c->M * sizeof(float), cudaMemcpyDeviceToDevice, st));
  return HOT_OK;
}

int restore_state(hot_ctx *c, const Saved &s, cudaStream_t st) {
  c->u_valid = false;
  HOT_CUDA(cudaMemcpyAsync(c->phi, s.phi, (size_t)c->W * c->H * sizeof(float), cudaMemcpyDeviceToDevice, st));
  HOT_CUDA(cudaMemcpyAsync(c->w, s.w, c->M * sizeof(float), cudaMemcpyDeviceToDevice, st));
  return HOT_OK;
}

// Best of three timed runs after one untimed run (graph capture, warm-up), in microseconds
// per iteration; restore() is queued before each run, outside the timed events.
template <typename Restore, typename Run>
int time_runs(cudaStream_t st, int iters, double *us, Restore restore, Run run) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HOT_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(HOT_ECUDA, "autotune: cudaEventCreate failed");
  }
  double best = 1e300;
  int rc = HOT_OK;
  for (int r = 0; rc == HOT_OK && r < 4; r++) {
    rc = restore();
    if (rc == HOT_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = fail(HOT_ECUDA, "autotune: event record failed");
    if (rc == HOT_OK) rc = run();
    if (rc == HOT_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = fail(HOT_ECUDA, "autotune: event record failed");
    float ms = 0.f;
    if (rc == HOT_OK) {
      cudaError_t e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) rc = fail(HOT_ECUDA, "autotune: %s", cudaGetErrorString(e));
    }
    if (rc == HOT_OK && r > 0) best = std::min(best, (double)ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == HOT_OK) *us = best * 1000.0 / iters;
  return rc;
}

}  // namespace

extern "C" {

int hot_set_tiling(hot_ctx *c, int rows, int blocks_per_sm, int chunk) {
  if (!c) return fail(HOT_EINVAL, "hot_set_tiling: NULL context");
  int rc = check_tiling("hot_set_tiling", rows, blocks_per_sm, chunk);
  if (rc != HOT_OK) return rc;
  HOT_CUDA(cudaStreamSynchronize(c->st));
  c->tile_rows = rows ? rows : hot::kRowsMax;
  c->tile_bps = blocks_per_sm;
  c->tile_chunk = chunk ? chunk : hot::kChunk;
  drop_graphs(c);
  return c->M ? build_schedule(c) : HOT_OK;
}

int hot_get_tiling(const hot_ctx *c, int *rows, int *blocks_per_sm, int *chunk) {
  if (!c) return fail(HOT_EINVAL, "hot_get_tiling: NULL context");
  if (rows) *rows = c->tile_rows;
  if (blocks_per_sm) *blocks_per_sm = c->sched_bps;
  if (chunk) *chunk = c->tile_chunk;
  return HOT_OK;
}

int hot_set_block_merge(hot_ctx *c, int merge) {
  if (!c) return fail(HOT_EINVAL, "hot_set_block_merge: NULL context");
  if (merge != 1 && merge != 2 && merge != 4) return fail(HOT_EINVAL, "hot_set_block_merge: merge = %d is not 1, 2 or 4", merge);
  HOT_CUDA(cudaStreamSynchronize(c->st));
  c->tile_merge = merge;
  drop_graphs(c);
  return c->M ? build_schedule(c) : HOT_OK;
}

int hot_get_block_merge(const hot_ctx *c, int *requested, int *in_effect) {
  if (!c) return fail(HOT_EINVAL, "hot_get_block_merge: NULL context");
  if (requested) *requested = c->tile_merge;
  if (in_effect) *in_effect = c->groups;
  return HOT_OK;
}

int hot_set_once(hot_ctx *c, int on) {
  if (!c) return fail(HOT_EINVAL, "hot_set_once: NULL context");
  if (on != 0 && on != 1) return fail(HOT_EINVAL, "hot_set_once: on = %d is not 0 or 1", on);
  HOT_CUDA(cudaStreamSynchronize(c->st));
  c->once_req = on != 0;
  c->u_valid = false;
  drop_graphs(c);
  return c->M ? build_schedule(c) : HOT_OK;
}

int hot_get_once(const hot_ctx *c, int *requested, int *in_effect) {
  if (!c) return fail(HOT_EINVAL, "hot_get_once: NULL context");
  if (requested) *requested = c->once_req ? 1 : 0;
  if (in_effect) *in_effect = c->once ? 1 : 0;
  return HOT_OK;
}

int hot_autotune(hot_ctx *c, int iters, int *rows, int *blocks_per_sm, int *chunk, double *us_per_iter) {
  if (!c) return fail(HOT_EINVAL, "hot_autotune: NULL context");
  if (!c->M) return fail(HOT_ESTATE, "hot_autotune: no traps set");
  if (iters < 1) return fail(HOT_EINVAL, "hot_autotune: iters = %d < 1", iters);
  if (c->precision == HOT_PREC_TENSOR)
    return fail(HOT_EINVAL, "hot_autotune: HOT_PREC_TENSOR has no tiling parameters (its tiles are fixed)");
  Saved saved;
  int rc = save_state(c, saved, c->st);
  if (rc != HOT_OK) return rc;
  const bool profiling = c->profiling;
  c->profiling = false;
  auto timed_gsw = [&](double *us) {
    return time_runs(c->st, iters, us, [&]() { return restore_state(c, saved, c->st); },
                     [&]() { return hot_gsw(c, iters, nullptr, nullptr); });
  };
  // The one-exponential step, where it applies, against the best tiling of the direct kernels
  // (which also serve the adjoint and the superposition).
  const bool once_req = c->once_req;
  double once_us = 0;
  if (once_req && c->once) {
    rc = timed_gsw(&once_us);
    if (rc == HOT_OK) rc = hot_set_once(c, 0);
  }
  Tiling best = {c->tile_rows, c->sched_bps, c->tile_chunk, c->tile_merge};
  double best_us = 0;
  if (rc == HOT_OK) rc = tune_tiling(
      kMaxBlocksPerSm, best, best_us,
      [&](const Tiling &t) {
        c->tile_merge = t.merge;  // applied by the schedule that hot_set_tiling rebuilds
        return hot_set_tiling(c, t.rows, t.bps, t.chunk);
      },
      timed_gsw, !separable_kernels(c));
  if (rc == HOT_OK && once_req && once_us > 0 && once_us < best_us) {
    rc = hot_set_once(c, 1);
    best_us = once_us;
  } else if (once_req && once_us > 0) {
    c->once_req = false;  // the direct kernels were faster (hot_get_once reports it)
  } else if (rc != HOT_OK) {
    c->once_req = once_req;
  }
  c->profiling = profiling;
  const int rc2 = restore_state(c, saved, c->st);
  cudaStreamSynchronize(c->st);
  c->have_fields = false;
  c->u_valid = false;
  if (rc != HOT_OK) return rc;
  if (rc2 != HOT_OK) return rc2;
  if (rows) *rows = best.rows;
  if (blocks_per_sm) *blocks_per_sm = best.bps;
  if (chunk) *chunk = best.chunk;
  if (us_per_iter) *us_per_iter = best_us;
  return HOT_OK;
}

int hot_batch_create(hot_batch **out, int count, hot_ctx *const *ctxs, void *cuda_stream) {
  if (!out) return fail(HOT_EINVAL, "hot_batch_create: out is NULL");
  *out = nullptr;
  if (count < 1 || !ctxs) return fail(HOT_EINVAL, "hot_batch_create: no contexts");
  for (int i = 0; i < count; i++) {
    if (!ctxs[i]) return fail(HOT_EINVAL, "hot_batch_create: context %d is NULL", i);
    if (!ctxs[i]->M) return fail(HOT_ESTATE, "hot_batch_create: context %d has no traps", i);
    if (ctxs[i]->precision != ctxs[0]->precision)
      return fail(HOT_EINVAL, "hot_batch_create: contexts differ in precision mode");
    if (ctxs[i]->H_total != ctxs[i]->H)
      return fail(HOT_EINVAL, "hot_batch_create: context %d is a row band (its sums need an exchange)", i);
    if (ctxs[i]->dev != ctxs[0]->dev) return fail(HOT_EINVAL, "hot_batch_create: contexts on different devices");
    for (int j = 0; j < i; j++)
      if (ctxs[j] == ctxs[i]) return fail(HOT_EINVAL, "hot_batch_create: context %d given twice", i);
  }
  hot_batch *b = new (std::nothrow) hot_batch;
  if (!b) return fail(HOT_ENOMEM, "hot_batch_create: out of host memory");
  b->count = count;
  b->ctx.assign(ctxs, ctxs + count);
  b->st = static_cast<cudaStream_t>(cuda_stream);
  b->precision = ctxs[0]->precision;
  b->dev = ctxs[0]->dev;
  const bool tensor = b->precision == HOT_PREC_TENSOR;
  int rc = tensor                                     ? HOT_OK
           : batch_mode(b) == hot::kModeSeparable ? batch_set_smem<hot::kModeSeparable>()
           : batch_mode(b) == hot::kModeFast      ? batch_set_smem<hot::kModeFast>()
                                                  : batch_set_smem<hot::kModeAccurate>();
  if (rc == HOT_OK && cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev) != cudaSuccess)
    rc = fail(HOT_ECUDA, "hot_batch_create: device query failed");
  if (rc == HOT_OK) rc = dalloc(&b->stamps, (size_t)count + 1);
  if (rc == HOT_OK) rc = tensor ? batch_setup_tensor(b) : batch_schedule(b);
  if (rc != HOT_OK) {
    batch_free(b);
    delete b;
    return rc;
  }
  *out = b;
  return HOT_OK;
}

int hot_batch_set_tiling(hot_batch *b, int rows, int blocks_per_sm, int chunk, double group_pairs) {
  if (!b) return fail(HOT_EINVAL, "hot_batch_set_tiling: NULL batch");
  if (b->precision == HOT_PREC_TENSOR) return fail(HOT_EINVAL, "hot_batch_set_tiling: a HOT_PREC_TENSOR batch has no tiling");
  int rc = check_tiling("hot_batch_set_tiling", rows, blocks_per_sm, chunk);
  if (rc != HOT_OK) return rc;
  if (!(group_pairs >= 0) || !std::isfinite(group_pairs))
    return fail(HOT_EINVAL, "hot_batch_set_tiling: group_pairs must be finite and >= 0");
  b->rows = rows ? rows : hot::kRowsMax;
  b->bps = blocks_per_sm;
  b->chunk = chunk ? chunk : hot::kChunk;
  b->group_pairs = group_pairs > 0 ? group_pairs : 67108864.0;
  return batch_schedule(b);
}

int hot_batch_get_tiling(const hot_batch *b, int *rows, int *blocks_per_sm, int *chunk, double *group_pairs,
                         int *groups) {
  if (!b) return fail(HOT_EINVAL, "hot_batch_get_tiling: NULL batch");
  if (rows) *rows = b->rows;
  if (blocks_per_sm) *blocks_per_sm = b->bps > 0 ? std::min(b->bps, b->per_sm_max) : b->per_sm_max;
  if (chunk) *chunk = b->chunk;
  if (group_pairs) *group_pairs = b->group_pairs;
  if (groups) *groups = (int)(b->precision == HOT_PREC_TENSOR ? b->chains.size() : b->groups.size());
  return HOT_OK;
}

int hot_batch_gsw(hot_batch *b, int iters) {
  if (!b) return fail(HOT_EINVAL, "hot_batch_gsw: NULL batch");
  if (iters < 0) return fail(HOT_EINVAL, "hot_batch_gsw: iters = %d < 0", iters);
  for (auto &g : b->graphs)
    if (g.iters == iters) {
      HOT_CUDA(cudaGraphLaunch(g.exec, b->st));
      for (auto *c : b->ctx) {
        c->have_fields = true;
        c->u_valid = false;  // the batch kernels wrote the phases
      }
      b->ran = true;
      return HOT_OK;
    }
  if (!b->cap) HOT_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  if (b->graphs.size() >= 8) {
    cudaGraphExecDestroy(b->graphs.front().exec);
    b->graphs.erase(b->graphs.begin());
  }
  cudaStream_t user = b->st;
  HOT_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  b->st = b->cap;
  int rc = batch_enqueue(b, iters);
  b->st = user;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
  if (rc != HOT_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(HOT_ECUDA, "hot_batch_gsw: graph capture: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(HOT_ECUDA, "hot_batch_gsw: graph instantiation: %s", cudaGetErrorString(e));
  b->graphs.push_back({iters, exec});
  HOT_CUDA(cudaGraphLaunch(exec, b->st));
  for (auto *c : b->ctx) {
    c->have_fields = true;
    c->u_valid = false;  // the batch kernels wrote the phases
  }
  b->ran = true;
  return HOT_OK;
}

int hot_batch_autotune(hot_batch *b, int iters, int *rows, int *blocks_per_sm, int *chunk, double *us_per_iter) {
  if (!b) return fail(HOT_EINVAL, "hot_batch_autotune: NULL batch");
  if (b->precision == HOT_PREC_TENSOR) return fail(HOT_EINVAL, "hot_batch_autotune: a HOT_PREC_TENSOR batch has no tiling");
  if (iters < 1) return fail(HOT_EINVAL, "hot_batch_autotune: iters = %d < 1", iters);
  std::vector<Saved> saved(b->count);
  int rc = HOT_OK;
  for (int h = 0; rc == HOT_OK && h < b->count; h++) rc = save_state(b->ctx[h], saved[h], b->st);
  if (rc != HOT_OK) return rc;
  auto restore = [&]() {
    for (int h = 0; h < b->count; h++) {
      const int r = restore_state(b->ctx[h], saved[h], b->st);
      if (r != HOT_OK) return r;
    }
    return (int)HOT_OK;
  };
  Tiling best = {b->rows, b->bps > 0 ? std::min(b->bps, b->per_sm_max) : b->per_sm_max, b->chunk, 1};
  double best_us = 0;
  const double gp = b->group_pairs;
  rc = tune_tiling(
      kMaxBlocksPerSm, best, best_us, [&](const Tiling &t) { return hot_batch_set_tiling(b, t.rows, t.bps, t.chunk, gp); },
      [&](double *us) { return time_runs(b->st, iters, us, restore, [&]() { return hot_batch_gsw(b, iters); }); });
  const int rc2 = restore();
  cudaStreamSynchronize(b->st);
  for (auto *c : b->ctx) {
    c->have_fields = false;
    c->u_valid = false;
  }
  b->ran = false;
  if (rc != HOT_OK) return rc;
  if (rc2 != HOT_OK) return rc2;
  if (rows) *rows = best.rows;
  if (blocks_per_sm) *blocks_per_sm = best.bps;
  if (chunk) *chunk = best.chunk;
  if (us_per_iter) *us_per_iter = best_us;
  return HOT_OK;
}

int hot_batch_latency(hot_batch *b, double *ms, int count) {
  if (!b || !ms) return fail(HOT_EINVAL, "hot_batch_latency: NULL argument");
  if (count != b->count) return fail(HOT_EINVAL, "hot_batch_latency: count = %d, the batch has %d", count, b->count);
  if (!b->ran) return fail(HOT_ESTATE, "hot_batch_latency: no hot_batch_gsw since the batch was (re)scheduled");
  std::vector<unsigned long long> t(count + 1);
  HOT_CUDA(cudaMemcpyAsync(t.data(), b->stamps, sizeof(unsigned long long) * (count + 1), cudaMemcpyDeviceToHost, b->st));
  HOT_CUDA(cudaStreamSynchronize(b->st));
  for (int h = 0; h < count; h++) ms[h] = (double)(long long)(t[h] - t[count]) * 1e-6;
  return HOT_OK;
}

void hot_batch_destroy(hot_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->st);
  batch_free(b);
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// SFU throughput probe (hot_sfu_rate).
namespace {

template <int OP>
__global__ void __launch_bounds__(1024) sfu_rate_kernel(float *out, long long *cycles, int iters, float step) {
  float acc[8], x[8];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    x[i] = 0.37f * i + 1e-3f * (threadIdx.x & 63) - 3.0f;
    acc[i] = 0.f;
  }
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) {
      if (OP != 3) x[i] += step;  // a new argument every iteration
      if (OP == 0) {
        acc[i] = fmaf(hot::sin_approx(x[i]), hot::cos_approx(x[i]), acc[i]);
      } else if (OP == 1) {
        acc[i] += hot::sin_approx(x[i]);
      } else if (OP == 2) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[i] * 0.001f));
        acc[i] += y;
      } else {
        acc[i] = fmaf(acc[i], 0.999f, x[i]);  // FP32 FMA pipe: 8 independent chains
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; i++) s += acc[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" int hot_tc_shape(int width, int height, int M, int sms, int *shape) {
  if (width < 1 || height < 1 || M < 1 || sms < 1 || !shape)
    return fail(HOT_EINVAL, "hot_tc_shape: invalid argument");
  const hot_tc::Shape sh = hot_tc::shape_for(width, height, M, sms);
  const int v[9] = {sh.bn_back, sh.bn_fwd, sh.fwd_splits, sh.fwd_cps, sh.Kb, sh.Kf, sh.rows_h, sh.rows_b, sh.rows_f};
  for (int i = 0; i < 9; i++) shape[i] = v[i];
  return HOT_OK;
}

extern "C" int hot_tc_gemm(int rows, int cols, int K, const float *A, const float *B, float *C, int tile_n,
                           int operands, void *cuda_stream) {
  if (rows < 1 || cols < 1 || K < 1) return fail(HOT_EINVAL, "hot_tc_gemm: sizes %d x %d x %d", rows, cols, K);
  if (!A || !B || !C) return fail(HOT_EINVAL, "hot_tc_gemm: NULL argument");
  if (tile_n != 32 && tile_n != 64 && tile_n != 128 && tile_n != 256)
    return fail(HOT_EINVAL, "hot_tc_gemm: tile_n = %d not 32, 64, 128 or 256", tile_n);
  if (operands != HOT_TC_TF32 && operands != HOT_TC_FP16)
    return fail(HOT_EINVAL, "hot_tc_gemm: operands = %d not HOT_TC_TF32 or HOT_TC_FP16", operands);
  if ((long long)rows * K >= (1LL << 31) || (long long)cols * K >= (1LL << 31) || (long long)rows * cols >= (1LL << 31))
    return fail(HOT_EINVAL, "hot_tc_gemm: operands of 2^31 elements or more");
  int timed_out = 0;
  const char *what = "";
  const cudaError_t e = hot_tc::gemm(rows, cols, K, A, B, C, tile_n, operands == HOT_TC_FP16 ? 1 : 0,
                                     static_cast<cudaStream_t>(cuda_stream), &timed_out, &what);
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? HOT_ENOMEM : HOT_ECUDA, "hot_tc_gemm: %s: %s", what,
                cudaGetErrorString(e));
  if (timed_out) return fail(HOT_ETIMEOUT, "hot_tc_gemm: a bounded device-side wait ran out");
  return HOT_OK;
}

extern "C" int hot_sfu_rate(int op, double *per_clk_per_sm, int *sms) {
  if (!per_clk_per_sm || op < 0 || op > 3) return fail(HOT_EINVAL, "hot_sfu_rate: invalid argument");
  int dev = 0, n = 0;
  HOT_CUDA(cudaGetDevice(&dev));
  HOT_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 1024, iters = 2048;
  float *out = nullptr;
  long long *cyc = nullptr;
  int rc = dalloc(&out, (size_t)n * threads);
  if (rc == HOT_OK) rc = dalloc(&cyc, (size_t)n);
  std::vector<long long> h(n);
  for (int rep = 0; rc == HOT_OK && rep < 2; rep++) {  // the first run warms up
    if (op == 0) sfu_rate_kernel<0><<<n, threads>>>(out, cyc, iters, 1e-4f);
    else if (op == 1) sfu_rate_kernel<1><<<n, threads>>>(out, cyc, iters, 1e-4f);
    else if (op == 2) sfu_rate_kernel<2><<<n, threads>>>(out, cyc, iters, 1e-4f);
    else sfu_rate_kernel<3><<<n, threads>>>(out, cyc, iters, 1e-4f);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, sizeof(long long) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = fail(HOT_ECUDA, "hot_sfu_rate: %s", cudaGetErrorString(e));
  }
  dfree(out);
  dfree(cyc);
  if (rc != HOT_OK) return rc;
  double mean = 0.0;
  for (long long v : h) mean += (double)v;
  mean /= n;
  const double results = (op == 0 ? 2.0 : 1.0) * threads * (double)iters * 8;  // per block (= per SM)
  *per_clk_per_sm = results / mean;
  if (sms) *sms = n;
  return HOT_OK;
}

// ---------------------------------------------------------------------------------------------
// Allocation-free trap-field evaluation (hot_field_noalloc): all working memory is carved out
// of one file-scope device array, whose device address is looked up once per device.
namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[HOT_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;

// What the first call on a device sets up: the scratch array's device address, the
// step kernels' shared-memory limit and the resident blocks per SM of the work schedule.
struct NoallocDevice {
  unsigned char *base;  // NULL until set up
  int sms, per_sm;
};
std::mutex g_noalloc_mutex;
NoallocDevice g_noalloc_dev[kNoallocMaxDevices];

// Set-up of device dev (the current device), once: the device address of the scratch array
// (in host code its name is a host-side stand-in, not a device address), the dynamic
// shared-memory limit of the forward-field kernels and the occupancy that sizes the grid
// (the same per-SM block count a context's schedule uses; it does not depend on M).
int noalloc_device(int dev, NoallocDevice *out) {
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(HOT_EINVAL, "hot_field_noalloc: device %d beyond %d", dev, kNoallocMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoallocDevice &d = g_noalloc_dev[dev];
  if (!d.base) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(HOT_ECUDA, "hot_field_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    const int fwd = hot::step_smem_bytes(1, false), step = hot::step_smem_bytes(1, true);
    HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fwd));
    HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fwd));
    HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, step));
    int sms = 0, per_sm = 0;
    HOT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hot::gsw_step_kernel<true, true, true>, hot::kThreads, step));
    d.sms = sms;
    d.per_sm = per_sm < 1 ? 1 : per_sm;
    d.base = static_cast<unsigned char *>(p);
  }
  *out = d;
  return HOT_OK;
}

// Number of sub-tiles block b of G receives: its run of the U = strips x H row segments,
// cut at strip ends and into pieces of at most kRowsMax rows (the rule of build_schedule).
__host__ __device__ int noalloc_block_subtiles(long long U, int G, int H, int b, hot::SubTile *out) {
  long long s = U * b / G;
  const long long s1 = U * (b + 1) / G;
  int n = 0;
  while (s < s1) {
    const int strip = (int)(s / H), row = (int)(s % H);
    const long long run_end = (s1 < (long long)(strip + 1) * H) ? s1 : (long long)(strip + 1) * H;
    const int L = (int)(run_end - s);
    const int nsub = (L + hot::kRowsMax - 1) / hot::kRowsMax;
    for (int i = 0; out && i < nsub; i++) {
      const int r0 = row + (int)((long long)L * i / nsub), r1 = row + (int)((long long)L * (i + 1) / nsub);
      out[n + i] = {strip * hot::kTileW, r0, r1 - r0, 0};
    }
    n += nsub;
    s = run_end;
  }
  return n;
}

// Writes the schedule (sub-tiles and per-block first index) for G blocks.
__global__ void noalloc_schedule_kernel(long long U, int G, int H, hot::SubTile *sub, int *first) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > G) return;
  int f = 0;
  for (int q = 0; q < b; q++) f += noalloc_block_subtiles(U, G, H, q, nullptr);
  first[b] = f;
  if (b < G) noalloc_block_subtiles(U, G, H, b, sub + f);
}

// a_m, b_m, c_m of Eq. 2 in turns per pixel index, from device trap coordinates.
__global__ void noalloc_abc_kernel(int M, const double *xyz, double lin, double quad, double *abc) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < M) {
    abc[3 * m] = xyz[3 * m] * lin;
    abc[3 * m + 1] = xyz[3 * m + 1] * lin;
    abc[3 * m + 2] = xyz[3 * m + 2] * quad;
  }
}

// Fixed-point field sums and metrics of the step kernel -> the caller's double outputs.
__global__ void noalloc_out_kernel(int M, const long long *Vsum, float, int width, int height, int fx_shift,
                                   const float *metrics, double *V, double *eu) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const double inv = 1.0 / ((double)width * (double)height * ldexp(1.0, fx_shift));
  if (m < M) {
    V[2 * m] = (double)Vsum[m] * inv;
    V[2 * m + 1] = (double)Vsum[M + m] * inv;
  }
  if (eu && m == 0) {
    eu[0] = metrics[0];
    eu[1] = metrics[1];
  }
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

extern "C" int hot_field_noalloc(int width, int height, double pitch_m, double wavelength_m, double focal_m,
                                 int M, const double *xyz_m, const float *phi, int precision, double *V,
                                 double *eu, void *cuda_stream) {
  if (width < 1 || height < 1 || (long long)width * height >= (1LL << 31))
    return fail(HOT_EINVAL, "hot_field_noalloc: invalid size %d x %d", width, height);
  if (!finite_pos(pitch_m) || !finite_pos(wavelength_m) || !finite_pos(focal_m))
    return fail(HOT_EINVAL, "hot_field_noalloc: pitch, wavelength and focal length must be finite and > 0");
  if (M < 1 || M > HOT_MAX_TRAPS) return fail(HOT_EINVAL, "hot_field_noalloc: M = %d not in [1, %d]", M, HOT_MAX_TRAPS);
  if (!xyz_m || !phi || !V) return fail(HOT_EINVAL, "hot_field_noalloc: NULL input or output");
  if (precision != HOT_PREC_ACCURATE && precision != HOT_PREC_FAST)
    return fail(HOT_EINVAL, "hot_field_noalloc: unknown precision %d", precision);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const bool fast = precision == HOT_PREC_FAST;
  int dev = 0;
  HOT_CUDA(cudaGetDevice(&dev));
  NoallocDevice d = {};
  int rc = noalloc_device(dev, &d);
  if (rc != HOT_OK) return rc;

  // Work schedule: identical to a context's (one wave of step-kernel blocks).
  const int strips = (width + hot::kTileW - 1) / hot::kTileW;
  const long long U = (long long)strips * height;
  const int G = (int)std::min<long long>((long long)d.sms * d.per_sm, U);
  int n_sub = 0;
  for (int b = 0; b < G; b++) n_sub += noalloc_block_subtiles(U, G, height, b, nullptr);

  // Carve the scratch array.
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += align256(bytes); return o; };
  const size_t o_abc = take(sizeof(double) * 3 * M);
  const size_t o_xt = take(sizeof(float) * (size_t)M * width), o_xr = take(sizeof(float) * (size_t)M * width);
  const size_t o_yt = take(sizeof(float) * (size_t)M * height), o_yr = take(sizeof(float) * (size_t)M * height);
  const size_t o_sub = take(sizeof(hot::SubTile) * n_sub), o_first = take(sizeof(int) * (G + 1));
  const size_t o_acc = take(sizeof(unsigned long long) * 6 * M), o_vsum = take(sizeof(long long) * 2 * M);
  const size_t o_met = take(sizeof(float) * 2);
  if (off > HOT_NOALLOC_SCRATCH_BYTES)
    return fail(HOT_EINVAL, "hot_field_noalloc: %d x %d pixels and %d traps need %zu bytes of scratch, the limit is %u",
                width, height, M, off, (unsigned)HOT_NOALLOC_SCRATCH_BYTES);
  unsigned char *const base = d.base;
  double *abc = reinterpret_cast<double *>(base + o_abc);
  float *Xt = reinterpret_cast<float *>(base + o_xt), *Xr = reinterpret_cast<float *>(base + o_xr);
  float *Yt = reinterpret_cast<float *>(base + o_yt), *Yr = reinterpret_cast<float *>(base + o_yr);
  hot::SubTile *d_sub = reinterpret_cast<hot::SubTile *>(base + o_sub);
  int *d_first = reinterpret_cast<int *>(base + o_first);
  unsigned long long *acc = reinterpret_cast<unsigned long long *>(base + o_acc);
  long long *Vsum = reinterpret_cast<long long *>(base + o_vsum);
  float *metrics = reinterpret_cast<float *>(base + o_met);

  // The schedule is written on the device; the accumulators start at zero (the array keeps
  // whatever the previous call left).
  noalloc_schedule_kernel<<<(G + 1 + 255) / 256, 256, 0, st>>>(U, G, height, d_sub, d_first);
  HOT_CUDA(cudaGetLastError());
  HOT_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 6 * M, st));

  const double lin = pitch_m / (wavelength_m * focal_m);
  const double quad = pitch_m * pitch_m / (2.0 * wavelength_m * focal_m * focal_m);
  noalloc_abc_kernel<<<(M + 255) / 256, 256, 0, st>>>(M, xyz_m, lin, quad, abc);
  HOT_CUDA(cudaGetLastError());
  const long long total = (long long)M * (width + height);
  const int tb = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  hot::build_tables_kernel<<<tb, 256, 0, st>>>(width, height, height, 0, M, abc, Xt, Yt, Xr, Yr, nullptr, nullptr);
  HOT_CUDA(cudaGetLastError());

  int bits = 0;
  while ((1LL << bits) < (long long)width * height) bits++;
  const int fx_shift = 61 - bits;
  hot::StepArgs a = {};  // the forward-only kernel reads no weights, coefficients or separable tables
  a.W = width;
  a.H = height;
  a.M = M;
  a.chunk = hot::kChunk;
  a.copies = 1;
  a.sub = d_sub;
  a.first = d_first;
  a.X = fast ? Xr : Xt;
  a.Y = fast ? Yr : Yt;
  a.phi = const_cast<float *>(phi);  // the forward-only kernel reads the phases and writes none
  a.acc_in = acc + 4 * (size_t)M;
  a.acc_out = acc;
  a.acc_clear = acc + 2 * (size_t)M;
  a.fx_scale = ldexpf(1.0f, fx_shift);
  a.inv_fx_n = (float)(1.0 / ((double)width * (double)height * ldexp(1.0, fx_shift)));
  a.angle_units = fast ? 1.0f : 0.15915494309189535f;
  a.angle_eta = fast ? hot::kFastEta : 0.0f;
  const int smem = hot::step_smem_bytes(M, false);
  if (fast) hot::gsw_step_kernel<true, false, true><<<G, hot::kThreads, smem, st>>>(a);
  else hot::gsw_step_kernel<false, false, true><<<G, hot::kThreads, smem, st>>>(a);
  HOT_CUDA(cudaGetLastError());
  hot::FinalizeArgs f = {};  // no weights to move (w_src = w_dst = NULL), no completion stamp
  f.M = M;
  f.copies = 1;
  f.acc = acc;
  f.acc_all = acc;
  f.Vsum = Vsum;
  f.metrics = metrics;
  f.inv_fx_n = a.inv_fx_n;
  hot::gsw_finalize_kernel<<<1, hot::kFinalizeThreads, 0, st>>>(f);
  HOT_CUDA(cudaGetLastError());
  noalloc_out_kernel<<<(M + 255) / 256, 256, 0, st>>>(M, Vsum, a.inv_fx_n, width, height, fx_shift, metrics, V, eu);
  HOT_CUDA(cudaGetLastError());
  return HOT_OK;
}
