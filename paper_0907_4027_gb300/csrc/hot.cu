// hot.cu -- host runtime and C ABI (include/hot.h) of the GSW hologram engine.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/hot.h"
#include "gsw_kernels.cuh"

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
  double pitch = 0, lam = 0, focal = 0;
  cudaStream_t st = nullptr;
  int dev = 0;
  int precision = HOT_PREC_ACCURATE;
  // work schedule of the step kernels (see hot::SubTile)
  int grid = 0, n_sub = 0;
  hot::SubTile *sub = nullptr;  // [n_sub]
  int *first = nullptr;         // [grid + 1]
  int sched_smem_M = -1;        // M the schedule's occupancy was computed for
  // state
  float *phi = nullptr;  // [N]
  int M = 0;
  double *abc = nullptr;                                       // [M][3]
  float *Xt = nullptr, *Yt = nullptr, *Xr = nullptr, *Yr = nullptr;  // tables
  float *w = nullptr;                                          // [2][M] weights (home: w[0])
  unsigned long long *acc = nullptr;                           // [3][2][M] fixed-point field sums
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
    long long kernels;
    cudaGraphExec_t exec;
  };
  bool use_graphs = true;
  cudaStream_t cap = nullptr;  // capture stream (capture is not allowed on the legacy stream)
  std::vector<Graph> graphs;
};

namespace {

bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

void drop_graphs(hot_ctx *c) {
  for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

void free_traps(hot_ctx *c) {
  drop_graphs(c);
  dfree(c->abc);
  dfree(c->Xt);
  dfree(c->Yt);
  dfree(c->Xr);
  dfree(c->Yr);
  dfree(c->w);
  dfree(c->acc);
  dfree(c->Vsum);
  c->M = 0;
  c->have_fields = false;
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
template <bool FAST, bool BACK, bool FWD, bool ADJ = false>
int launch_tile(hot_ctx *c, bool pdl, int k, const float *phi = nullptr, const float2 *G = nullptr,
                float *grad = nullptr) {
  hot::StepArgs a;
  a.W = c->W;
  a.H = c->H;
  a.M = c->M;
  a.sub = c->sub;
  a.first = c->first;
  a.X = FAST ? c->Xr : c->Xt;
  a.Y = FAST ? c->Yr : c->Yt;
  a.phi = c->phi;
  const size_t M2 = 2 * (size_t)c->M;
  a.acc_in = c->acc + M2 * ((k + 2) % 3);
  a.acc_out = c->acc + M2 * (k % 3);
  a.acc_clear = c->acc + M2 * ((k + 1) % 3);
  a.w_in = c->w + (size_t)c->M * ((k + 1) & 1);
  a.w_out = c->w + (size_t)c->M * (k & 1);
  a.fx_scale = ldexpf(1.0f, c->fx_shift);
  a.inv_fx_n = (float)(1.0 / ((double)c->W * (double)c->H * ldexp(1.0, c->fx_shift)));
  a.angle_units = FAST ? 1.0f : 0.15915494309189535f;
  if (phi) a.phi = const_cast<float *>(phi);  // read only: forward field or adjoint of given phases
  a.G = G;
  a.grad = grad;
  a.inv_n = (float)(1.0 / ((double)c->W * (double)c->H));
  const int smem = hot::step_smem_bytes(c->M, BACK);
  Probe p(c, BACK && FWD ? HOT_KERNEL_STEP : FWD ? HOT_KERNEL_FORWARD : HOT_KERNEL_OTHER);
  launch(c, hot::gsw_step_kernel<FAST, BACK, FWD, ADJ>, c->grid, hot::kThreads, smem, pdl, a);
  return check_launch(c, "gsw_step_kernel");
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
  return HOT_OK;
}

// One wave of persistent blocks (SMs x resident blocks of the fused kernel); the W/32 x H row
// segments are dealt out in equal contiguous runs, cut into sub-tiles of <= kRowsMax rows.
int build_schedule(hot_ctx *c) {
  int rc = set_step_smem(c->M);
  if (rc != HOT_OK) return rc;
  int sms = 0, per_sm = 0;
  HOT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
  HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hot::gsw_step_kernel<true, true, true>,
                                                         hot::kThreads, hot::step_smem_bytes(c->M, true)));
  if (per_sm < 1) per_sm = 1;
  const int strips = (c->W + hot::kTileW - 1) / hot::kTileW;
  const long long U = (long long)strips * c->H;
  const int G = (int)std::min<long long>((long long)sms * per_sm, U);
  std::vector<hot::SubTile> sub;
  std::vector<int> first(G + 1);
  for (int b = 0; b < G; b++) {
    first[b] = (int)sub.size();
    long long s = U * b / G;
    const long long s1 = U * (b + 1) / G;
    while (s < s1) {
      const int strip = (int)(s / c->H), row = (int)(s % c->H);
      const long long run_end = std::min<long long>(s1, (long long)(strip + 1) * c->H);
      const int L = (int)(run_end - s);
      const int nsub = (L + hot::kRowsMax - 1) / hot::kRowsMax;
      for (int i = 0; i < nsub; i++) {
        const int r0 = row + (int)((long long)L * i / nsub), r1 = row + (int)((long long)L * (i + 1) / nsub);
        sub.push_back({strip * hot::kTileW, r0, r1 - r0, 0});
      }
      s = run_end;
    }
  }
  first[G] = (int)sub.size();
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
  return HOT_OK;
}

// One step-kernel launch (launch k of the sequence): weight update + back-projection and/or
// forward field.
int launch_step(hot_ctx *c, bool back, bool fwd, bool pdl, int k) {
  const bool fast = c->precision == HOT_PREC_FAST;
  if (back && fwd) return fast ? launch_tile<true, true, true>(c, pdl, k) : launch_tile<false, true, true>(c, pdl, k);
  if (back) return fast ? launch_tile<true, true, false>(c, pdl, k) : launch_tile<false, true, false>(c, pdl, k);
  return fast ? launch_tile<true, false, true>(c, pdl, k) : launch_tile<false, false, true>(c, pdl, k);
}

// After the last launch (k = iters): Eq. 4 metrics, field sums, weights home, accumulators cleared.
int launch_finalize(hot_ctx *c, bool pdl, int iters) {
  hot::FinalizeArgs f;
  const size_t M2 = 2 * (size_t)c->M;
  f.M = c->M;
  f.acc = c->acc + M2 * (iters % 3);
  f.acc_all = c->acc;
  f.w_src = c->w + (size_t)c->M * (iters & 1);
  f.w_dst = c->w;
  f.Vsum = c->Vsum;
  f.metrics = c->metrics;
  f.inv_fx_n = (float)(1.0 / ((double)c->W * (double)c->H * ldexp(1.0, c->fx_shift)));
  Probe p(c, HOT_KERNEL_FINISH);
  launch(c, hot::gsw_finalize_kernel, 1, hot::kFinalizeThreads, 0, pdl, f);
  return check_launch(c, "gsw_finalize_kernel");
}

// The launch sequence of hot_gsw(iters) on c->st.
// Inside the sequence every kernel is a programmatic dependent of the one before it (except
// when profiling, where events separate the launches); the first one waits normally for
// whatever preceded hot_gsw in the stream (trap tables, phases).
int enqueue_gsw(hot_ctx *c, int iters) {
  const bool pdl = !c->profiling;
  int rc = launch_step(c, false, true, false, 0);       // V^1 = F(phi^0)
  for (int k = 1; k <= iters && rc == HOT_OK; k++)
    rc = launch_step(c, true, true, pdl, k);            // w^k, c^k from V^k; phi^k; V^{k+1} = F(phi^k)
  if (rc == HOT_OK) rc = launch_finalize(c, pdl, iters);  // e, u of V^{iters+1}
  return rc;
}

// Replays (capturing on first use) the graph of enqueue_gsw(iters).
int launch_gsw_graph(hot_ctx *c, int iters) {
  for (auto &g : c->graphs)
    if (g.iters == iters && g.precision == c->precision) {
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
  c->graphs.push_back({iters, c->precision, kernels, exec});
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
  {  // fixed-point scale of the field sums: |sum| <= N, kept below 2^61
    int bits = 0;
    while ((1LL << bits) < (long long)width * height) bits++;
    c->fx_shift = 61 - bits;
  }
  int rc = HOT_OK;
  cudaError_t e = cudaGetDevice(&c->dev);
  if (e != cudaSuccess) rc = fail(HOT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  const size_t N = (size_t)width * height;
  if (rc == HOT_OK) rc = dalloc(&c->phi, N);
  if (rc == HOT_OK) rc = dalloc(&c->metrics, 2);
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
  dfree(c->metrics);
  dfree(c->u8);
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
    if (rc == HOT_OK) rc = dalloc(&c->w, 2 * (size_t)M);
    if (rc == HOT_OK) rc = dalloc(&c->acc, 6 * (size_t)M);
    if (rc == HOT_OK) rc = dalloc(&c->Vsum, 2 * (size_t)M);
    if (rc == HOT_OK && cudaMemsetAsync(c->acc, 0, sizeof(unsigned long long) * 6 * M, c->st) != cudaSuccess)
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
  const long long total = (long long)M * (c->W + c->H);
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  Probe p(c, HOT_KERNEL_OTHER);
  hot::build_tables_kernel<<<blocks, 256, 0, c->st>>>(c->W, c->H, M, c->abc, c->Xt, c->Yt, c->Xr, c->Yr);
  c->have_fields = false;
  return check_launch(c, "build_tables_kernel");
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
  return HOT_OK;
}

int hot_set_precision(hot_ctx *c, int precision) {
  if (!c) return fail(HOT_EINVAL, "hot_set_precision: NULL context");
  if (precision != HOT_PREC_ACCURATE && precision != HOT_PREC_FAST)
    return fail(HOT_EINVAL, "hot_set_precision: unknown mode %d", precision);
  c->precision = precision;
  return HOT_OK;
}

int hot_gsw(hot_ctx *c, int iters, double *eff_out, double *unif_out) {
  if (!c) return fail(HOT_EINVAL, "hot_gsw: NULL context");
  if (iters < 0) return fail(HOT_EINVAL, "hot_gsw: iters = %d < 0", iters);
  if (!c->M) return fail(HOT_ESTATE, "hot_gsw: no traps set");
  const int rc = (c->use_graphs && !c->profiling) ? launch_gsw_graph(c, iters) : enqueue_gsw(c, iters);
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
  std::vector<long long> vs(V ? 2 * c->M : 0);
  std::vector<float> wf(w ? c->M : 0);
  if (V) HOT_CUDA(cudaMemcpyAsync(vs.data(), c->Vsum, sizeof(long long) * 2 * c->M, cudaMemcpyDeviceToHost, c->st));
  if (w) HOT_CUDA(cudaMemcpyAsync(wf.data(), c->w, sizeof(float) * c->M, cudaMemcpyDeviceToHost, c->st));
  HOT_CUDA(cudaStreamSynchronize(c->st));
  const double inv = 1.0 / ((double)c->W * (double)c->H * ldexp(1.0, c->fx_shift));
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
  const bool fast = c->precision == HOT_PREC_FAST;
  int rc = fast ? launch_tile<true, false, true>(c, false, 0, phi) : launch_tile<false, false, true>(c, false, 0, phi);
  if (rc == HOT_OK) rc = launch_finalize(c, false, 0);  // w stays in w[0]; accumulators cleared
  if (rc != HOT_OK) return rc;
  const double inv = 1.0 / ((double)c->W * (double)c->H * ldexp(1.0, c->fx_shift));
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
    rc = c->precision == HOT_PREC_FAST ? launch_tile<true, true, false>(c, false, 0, nullptr, d)
                                       : launch_tile<false, true, false>(c, false, 0, nullptr, d);
  if (rc == HOT_OK) {
    e = cudaStreamSynchronize(c->st);  // the coefficients are freed below
    if (e != cudaSuccess) rc = fail(HOT_ECUDA, "hot_superposition: %s", cudaGetErrorString(e));
  }
  dfree(d);
  c->have_fields = false;
  return rc;
}

int hot_field_adjoint(hot_ctx *c, const float *phi, const float *G, float *grad) {
  if (!c || !phi || !G || !grad) return fail(HOT_EINVAL, "hot_field_adjoint: NULL argument");
  if (!c->M) return fail(HOT_ESTATE, "hot_field_adjoint: no traps set");
  const float2 *g = reinterpret_cast<const float2 *>(G);
  return c->precision == HOT_PREC_FAST ? launch_tile<true, true, false, true>(c, false, 0, phi, g, grad)
                                       : launch_tile<false, true, false, true>(c, false, 0, phi, g, grad);
}

int hot_sync(hot_ctx *c) {
  if (!c) return fail(HOT_EINVAL, "hot_sync: NULL context");
  HOT_CUDA(cudaStreamSynchronize(c->st));
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
      x[i] += step;  // a new argument every iteration
      if (OP == 0) {
        acc[i] = fmaf(hot::sin_approx(x[i]), hot::cos_approx(x[i]), acc[i]);
      } else if (OP == 1) {
        acc[i] += hot::sin_approx(x[i]);
      } else {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[i] * 0.001f));
        acc[i] += y;
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

extern "C" int hot_sfu_rate(int op, double *per_clk_per_sm, int *sms) {
  if (!per_clk_per_sm || op < 0 || op > 2) return fail(HOT_EINVAL, "hot_sfu_rate: invalid argument");
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
    else sfu_rate_kernel<2><<<n, threads>>>(out, cyc, iters, 1e-4f);
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
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_base[kNoallocMaxDevices];  // device address per device, or NULL

// Device address of the scratch array on the current device (looked up on first use).
int noalloc_scratch(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(HOT_EINVAL, "hot_field_noalloc: device %d beyond %d", dev, kNoallocMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_base[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(HOT_ECUDA, "hot_field_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_noalloc_base[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_noalloc_base[dev];
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

  // Work schedule: identical to a context's (one wave of step-kernel blocks).
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                hot::step_smem_bytes(M, false)));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                hot::step_smem_bytes(M, false)));
  HOT_CUDA(cudaFuncSetAttribute(hot::gsw_step_kernel<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                hot::step_smem_bytes(M, true)));
  int sms = 0, per_sm = 0;
  HOT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hot::gsw_step_kernel<true, true, true>,
                                                         hot::kThreads, hot::step_smem_bytes(M, true)));
  if (per_sm < 1) per_sm = 1;
  const int strips = (width + hot::kTileW - 1) / hot::kTileW;
  const long long U = (long long)strips * height;
  const int G = (int)std::min<long long>((long long)sms * per_sm, U);
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
  const size_t o_w = take(sizeof(float) * M), o_met = take(sizeof(float) * 2);
  if (off > HOT_NOALLOC_SCRATCH_BYTES)
    return fail(HOT_EINVAL, "hot_field_noalloc: %d x %d pixels and %d traps need %zu bytes of scratch, the limit is %u",
                width, height, M, off, (unsigned)HOT_NOALLOC_SCRATCH_BYTES);
  unsigned char *base = nullptr;
  int rc = noalloc_scratch(dev, &base);
  if (rc != HOT_OK) return rc;
  double *abc = reinterpret_cast<double *>(base + o_abc);
  float *Xt = reinterpret_cast<float *>(base + o_xt), *Xr = reinterpret_cast<float *>(base + o_xr);
  float *Yt = reinterpret_cast<float *>(base + o_yt), *Yr = reinterpret_cast<float *>(base + o_yr);
  hot::SubTile *d_sub = reinterpret_cast<hot::SubTile *>(base + o_sub);
  int *d_first = reinterpret_cast<int *>(base + o_first);
  unsigned long long *acc = reinterpret_cast<unsigned long long *>(base + o_acc);
  long long *Vsum = reinterpret_cast<long long *>(base + o_vsum);
  float *w = reinterpret_cast<float *>(base + o_w);
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
  hot::build_tables_kernel<<<tb, 256, 0, st>>>(width, height, M, abc, Xt, Yt, Xr, Yr);
  HOT_CUDA(cudaGetLastError());

  int bits = 0;
  while ((1LL << bits) < (long long)width * height) bits++;
  const int fx_shift = 61 - bits;
  hot::StepArgs a;
  a.W = width;
  a.H = height;
  a.M = M;
  a.sub = d_sub;
  a.first = d_first;
  a.X = fast ? Xr : Xt;
  a.Y = fast ? Yr : Yt;
  a.phi = const_cast<float *>(phi);  // the forward-only kernel reads the phases and writes none
  a.acc_in = acc + 4 * (size_t)M;
  a.acc_out = acc;
  a.acc_clear = acc + 2 * (size_t)M;
  a.w_in = w;
  a.w_out = w;
  a.fx_scale = ldexpf(1.0f, fx_shift);
  a.inv_fx_n = (float)(1.0 / ((double)width * (double)height * ldexp(1.0, fx_shift)));
  a.angle_units = fast ? 1.0f : 0.15915494309189535f;
  const int smem = hot::step_smem_bytes(M, false);
  if (fast) hot::gsw_step_kernel<true, false, true><<<G, hot::kThreads, smem, st>>>(a);
  else hot::gsw_step_kernel<false, false, true><<<G, hot::kThreads, smem, st>>>(a);
  HOT_CUDA(cudaGetLastError());
  hot::FinalizeArgs f;
  f.M = M;
  f.acc = acc;
  f.acc_all = acc;
  f.w_src = w;
  f.w_dst = w;
  f.Vsum = Vsum;
  f.metrics = metrics;
  f.inv_fx_n = a.inv_fx_n;
  hot::gsw_finalize_kernel<<<1, hot::kFinalizeThreads, 0, st>>>(f);
  HOT_CUDA(cudaGetLastError());
  noalloc_out_kernel<<<(M + 255) / 256, 256, 0, st>>>(M, Vsum, a.inv_fx_n, width, height, fx_shift, metrics, V, eu);
  HOT_CUDA(cudaGetLastError());
  return HOT_OK;
}
