// api.cu -- host implementation of the C ABI declared in rt.h.
#include <utility>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rt.h"
#include "healpix.cuh"
#include "policy.h"
#include "rt_internal.cuh"

namespace rtg {
cudaError_t launch_trace_init(unsigned long long* ctl, void* queue, size_t queue_bytes, unsigned long long n_roots,
                              int first_pass, int mode, unsigned long long in_cap, int pass, int passes,
                              cudaStream_t st);
cudaError_t trace_occupancy(int precision, int fsl, int block, int* blocks_per_sm);
cudaError_t launch_trace(int precision, int fsl, const TraceArgs& A, int grid, int block, cudaStream_t st);
cudaError_t launch_flight_table(const double* old, double* neu, float2* neu32, int n_new, double c_dt,
                                cudaStream_t st);

cudaError_t launch_chem(int precision, long long ncell, const double* nH, double* xHI, double* xHII,
                        const void* K, void* nhi, double h, int nsub, double alpha, cudaStream_t st);
cudaError_t launch_refresh(int precision, long long ncell, const double* nH, const double* xHI,
                           void* nhi, cudaStream_t st);
cudaError_t launch_convert(long long n, const void* src, int src_dtype, void* dst, int dst_dtype,
                           cudaStream_t st, double scale = 1.0);
cudaError_t launch_complement(long long n, const double* x, double* out, cudaStream_t st);
cudaError_t launch_commit_state(int precision, long long n, unsigned long long* ctl, const double* sn,
                               const double* sx, const double* sz, double* nH, double* xHI, double* xHII, void* nhi,
                               cudaStream_t st);
cudaError_t launch_timestep(long long n, int nx, int ny, int nz, const double* nH, const double* xHI, const void* K,
                            int fp64_rates, double sdx, double tau_front, float eps, float alpha, float dt_max,
                            float unit, float* dtc, unsigned int* out, cudaStream_t st);
cudaError_t launch_check_state(long long n, const double* nH, const double* x, unsigned long long* bad,
                               cudaStream_t st);
cudaError_t launch_check_density(long long n, const double* a, unsigned long long* bad, cudaStream_t st);
cudaError_t launch_add_word(unsigned long long* w, unsigned long long delta, cudaStream_t st);
cudaError_t launch_zero_fields(void* a, void* b, size_t nbytes, void* acc, int nacc, void* cnt, int ncnt,
                               cudaStream_t st);
cudaError_t launch_check_refresh(int precision, long long n, unsigned long long* ctl, const double* nH, double* x,
                                 double* z, int z_given, const double* x_old, const double* z_old, void* nhi,
                                 InstDev* inst, cudaStream_t st);
cudaError_t launch_pair(long long n, const double* src, void* dst, cudaStream_t st);
cudaError_t launch_direction_check(int level, unsigned long long* out, cudaStream_t st);
cudaError_t launch_direction_table(int level, float4* tab, cudaStream_t st);
cudaError_t launch_batch_zero(const InstDev* inst, int ninst, int precision, long long max_cells, cudaStream_t st);
cudaError_t launch_batch_chem(const InstDev* inst, int ninst, int precision, long long max_cells, double h,
                              int nsub, double alpha, cudaStream_t st);
}  // namespace rtg

using namespace rtg;

// A named range on the profiler's timeline (NVTX) for the duration of a call;
// free when no profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CUDA_TRY(call)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                         \
    }                                                                                         \
  } while (0)

#define LAUNCH_TRY(call)  \
  do {                    \
    CUDA_TRY(call);       \
    g_launches.fetch_add(1); \
  } while (0)

struct rt_ctx {
  int device;
  int num_sms;
  // pixel directions as FP32 pairs (mixed path), levels 0..dir_levels
  // Tables replaced by a deeper one stay allocated until the context is
  // destroyed: a trace enqueued from another thread may still hold them.
  std::mutex dir_mu;
  float4* dir_tab = nullptr;
  int dir_levels = -1;
  std::vector<float4*> dir_retired;
  ~rt_ctx() {
    if (dir_tab) cudaFree(dir_tab);
    for (float4* t : dir_retired) cudaFree(t);
  }
};

constexpr int kDirTableMaxLevel = 9;  // 4.2M pixels, 134 MB

// Make sure the direction table holds levels 0..want (want <= 9); the table
// and its deepest level are returned as read under the lock.
static int ensure_dir_table(rt_ctx* c, int want, const float4** tab, int* levels) {
  std::lock_guard<std::mutex> lk(c->dir_mu);
  if (want <= c->dir_levels) {
    *tab = c->dir_tab;
    *levels = c->dir_levels;
    return RT_OK;
  }
  const size_t entries = (size_t)4 * (((size_t)1 << (2 * (want + 1))) - 1);
  float4* t = nullptr;
  CUDA_TRY(cudaMalloc(&t, entries * 2 * sizeof(float4)));
  for (int l = 0; l <= want; ++l) {
    cudaError_t e = launch_direction_table(l, t, 0);
    if (e != cudaSuccess) { cudaFree(t); return fail(RT_ERR_CUDA, "direction table: %s", cudaGetErrorString(e)); }
    g_launches.fetch_add(1);
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { cudaFree(t); return fail(RT_ERR_CUDA, "direction table: %s", cudaGetErrorString(e)); }
  if (c->dir_tab) c->dir_retired.push_back(c->dir_tab);
  c->dir_tab = t;
  c->dir_levels = want;
  *tab = t;
  *levels = want;
  return RT_OK;
}

// Per-trace device resources: queue, control words, descriptors.
struct TraceState {
  void* queue = nullptr;
  unsigned long long cap = 0;  // records
  size_t rec_bytes = 0;
  unsigned long long* ctl = nullptr;
  double* blk = nullptr;  // per-block budget rows (allocated with the grid or batch)
  int blk_blocks = 0;     // blocks the rows are allocated for
  int blk_rows = 0;       // grids per block
  int passes = 1;       // source ranges the last automatically sized trace used
  int passes_run = 1;   // passes of the last trace launched
  ~TraceState() {
    if (queue) cudaFree(queue);
    if (ctl) cudaFree(ctl);
    if (blk) cudaFree(blk);
  }
  // Rows for `blocks` blocks of a launch over `ninst` grids.
  int bind_rows(TraceArgs& A, int blocks, int ninst) const {
    if (blocks > blk_blocks)
      return fail(RT_ERR_INVALID_ARG, "trace launch of %d blocks exceeds the %d blocks of its budget rows", blocks,
                  blk_blocks);
    A.blk = blk;
    A.blk_rows = ninst < blk_rows ? ninst : blk_rows;
    return RT_OK;
  }
};

constexpr int kAccWords = 8;  // photon budget sums per grid (see InstDev.acc)

// Packages in flight between traces (finite speed of light): two stores used
// alternately (the next trace continues what the last one halted into
// buf[in] and halts into the other), the halting radius per age on the
// device (double-buffered too), and, per source, the photon unit that the
// stored P values are expressed in.
struct FlightState {
  void* buf[2] = {nullptr, nullptr};
  unsigned long long cap[2] = {0, 0};
  int in = 0;                 // store holding the packages of the last trace
  bool live = false;          // the last trace halted packages into buf[in]
  int in_before = 0;          // in / live before the trace being run (a retry starts again from them)
  bool live_before = false;
  std::vector<double> rlim;   // halting radii of the last trace (host mirror)
  double* rlim64[2] = {nullptr, nullptr};
  float2* rlim32[2] = {nullptr, nullptr};
  size_t rlim_cap[2] = {0, 0};
  int tab = 0;                // device table holding rlim
  std::vector<double> pend;   // radii of the trace being launched (become rlim when it is)
  std::vector<double> unit;   // per source: photons/s of P = 1 for the stored packages
  unsigned long long last_halted = 0;  // packages halted by the last synchronous trace
  ~FlightState() {
    for (int i = 0; i < 2; ++i) {
      if (buf[i]) cudaFree(buf[i]);
      if (rlim64[i]) cudaFree(rlim64[i]);
      if (rlim32[i]) cudaFree(rlim32[i]);
    }
  }
};

struct rt_grid {
  rt_ctx* ctx;
  int nx, ny, nz;
  long long ncell;
  double box_len_cm, dx;
  int precision;
  cudaStream_t stream;
  double* nH = nullptr;
  double* xHI = nullptr;
  double* xHII = nullptr;
  void* nhi = nullptr;  // FP64 or FP32
  void* K = nullptr;
  void* G = nullptr;
  double* acc = nullptr;               // kAccWords doubles
  unsigned long long* cnt = nullptr;   // kCntWords
  InstDev* inst_dev = nullptr;
  struct SrcIn { double pos[3], ndot, e_ph, sigma; int type = 0; };
  // helium absorbers and rates of photon types 1 (He I) and 2 (He II), once set
  bool he = false;
  double* nhe64[2] = {nullptr, nullptr};
  void* nhe[2] = {nullptr, nullptr};  // FP64 grid: nhe64; FP32-mixed: FP32 pairs
  void* Khe[2] = {nullptr, nullptr};
  void* Ghe[2] = {nullptr, nullptr};
  std::vector<SrcIn> src;              // sources as given by the caller
  SourceDev* src_dev = nullptr;
  size_t src_dev_cap = 0;
  bool src_dirty = true;
  int last_level0 = -1;
  int src_offset = 0;                  // index of the first source in checksums
  TraceState ts;
  FlightState fl;
  bool src_fsl = false;                // the device source table was built for a finite-c trace
  double seg_per_pkg = 0.0;            // segments per package of the last trace read back
  // pinned readback buffer
  void* host_rb = nullptr;
  bool traced = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the last trace kernel
  rt_batch* batch = nullptr;                 // the batch holding the grid (at most one)
  int batch_slot = -1;
  cudaStream_t batch_stream = nullptr;       // set while the grid is in a batch
  // Uploads and read-backs that do not wait (rt_set_state_async,
  // rt_get_rates_async): host->device copies run on `up`, device->host copies
  // on `dn`, through library-owned staging areas, ordered against the grid's
  // stream by events; created on first use.
  cudaStream_t up = nullptr, dn = nullptr;
  cudaEvent_t ev_up = nullptr, ev_commit = nullptr, ev_snap = nullptr;
  cudaEvent_t ev_dl[3] = {nullptr, nullptr, nullptr};  // last host copy of each staged field
  double* up_stage = nullptr;                // 3 * ncell doubles: n_H, x_HI, x_HII
  double* xHI_alt = nullptr;                 // alternate state buffers: an upload without n_H goes
  double* xHII_alt = nullptr;                // into them and they swap with xHI, xHII on commit
  char* dn_stage = nullptr;                  // 3 * ncell * 8 bytes: k_ph, Gamma, x_HI
  std::string set_err;                       // message of a rejected asynchronous state
  bool check_words_set = false;              // CTL_CHECK_N/X hold ~0 (then kept so by each commit)
  ~rt_grid() {
    if (up) cudaStreamSynchronize(up);
    if (dn) cudaStreamSynchronize(dn);
    cudaFree(up_stage); cudaFree(dn_stage); cudaFree(xHI_alt); cudaFree(xHII_alt);
    for (cudaEvent_t ev : {ev_up, ev_commit, ev_snap, ev_dl[0], ev_dl[1], ev_dl[2]})
      if (ev) cudaEventDestroy(ev);
    if (up) cudaStreamDestroy(up);
    if (dn) cudaStreamDestroy(dn);
    cudaFree(nH); cudaFree(xHI); cudaFree(xHII); cudaFree(nhi); cudaFree(K); cudaFree(G);
    cudaFree(acc); cudaFree(cnt); cudaFree(inst_dev); cudaFree(src_dev);
    for (int t = 0; t < 2; ++t) {
      if (nhe[t] != nhe64[t]) cudaFree(nhe[t]);
      cudaFree(nhe64[t]); cudaFree(Khe[t]); cudaFree(Ghe[t]);
    }
    if (host_rb) cudaFreeHost(host_rb);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  }
};

static size_t elem_bytes(int precision) { return precision == RT_FP64 ? 8 : 4; }

// The trace kernel's view of a grid (slot `inst` of a launch).
static InstDev inst_of(const rt_grid* g) {
  InstDev I;
  memset(&I, 0, sizeof I);
  I.nx = g->nx; I.ny = g->ny; I.nz = g->nz;
  I.flags = g->precision == RT_FP32_MIXED ? kInstNhiPair : 0;
  I.nhi = g->nhi; I.nH = g->nH; I.xHI = g->xHI; I.xHII = g->xHII; I.K = g->K; I.G = g->G;
  I.acc = g->acc; I.cnt = g->cnt;
  for (int t = 0; t < 2; ++t) {
    I.nhe[t] = g->nhe[t]; I.nhe64[t] = g->nhe64[t]; I.Khe[t] = g->Khe[t]; I.Ghe[t] = g->Ghe[t];
  }
  return I;
}

// A grid in a batch is updated on the batch's stream: per-grid calls first
// wait for that work.
static int wait_batch(rt_grid* g) {
  if (g->batch_stream) CUDA_TRY(cudaStreamSynchronize(g->batch_stream));
  return RT_OK;
}

// Take a grid out of its batch; have its batch rebuild its tables before
// the next launch (both defined with the batches).
static void detach_grid(rt_grid* g);
static void mark_batch_dirty(rt_grid* g);

extern "C" {

const char* rt_get_last_error(void) { return g_last_error.c_str(); }

uint64_t rt_kernel_launches(void) { return g_launches.load(); }

int rt_ctx_create(int device, rt_ctx** out) {
  if (!out) return fail(RT_ERR_INVALID_ARG, "rt_ctx_create: out is NULL");
  int n = 0;
  CUDA_TRY(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(RT_ERR_INVALID_ARG, "rt_ctx_create: device %d of %d", device, n);
  CUDA_TRY(cudaSetDevice(device));
  int num_sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
  rt_ctx* c = new rt_ctx;
  c->device = device;
  c->num_sms = num_sms;
  *out = c;
  g_last_error.clear();
  return RT_OK;
}

int rt_ctx_destroy(rt_ctx* ctx) {
  delete ctx;
  return RT_OK;
}

// Range check of a state already on the device (nH may be NULL), on stream
// st: RT_OK, or RT_ERR_INVALID_ARG naming the first bad cell and its value.
// Synchronises st.
static int check_state(const char* who, long long ncell, const double* nH, const double* x, cudaStream_t st) {
  unsigned long long* bad = nullptr;
  CUDA_TRY(cudaMallocAsync((void**)&bad, 2 * sizeof(unsigned long long), st));
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaMemsetAsync(bad, 0xff, 2 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = launch_check_state(ncell, nH, x, bad, st);
  if (e == cudaSuccess) g_launches.fetch_add(1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, bad, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(bad, st);
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, "%s: state check: %s", who, cudaGetErrorString(e));
  for (int k = 0; k < 2; ++k) {
    if (h[k] == ~0ULL) continue;
    double v = 0.0;
    cudaMemcpy(&v, (k == 0 ? nH : x) + h[k], sizeof v, cudaMemcpyDeviceToHost);
    return fail(RT_ERR_INVALID_ARG, "%s: %s[%llu] = %g", who, k == 0 ? "n_H" : "x_HI", h[k], v);
  }
  return RT_OK;
}

static int upload(void* dst, const void* src, size_t bytes, int mem_kind, cudaStream_t st) {
  CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, mem_kind == RT_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                                        : cudaMemcpyHostToDevice, st));
  return RT_OK;
}

int rt_create_grid(rt_ctx* ctx, const rt_grid_desc* d, void* stream, rt_grid** out) {
  if (!ctx || !d || !out) return fail(RT_ERR_INVALID_ARG, "rt_create_grid: NULL argument");
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(RT_ERR_INVALID_ARG, "rt_create_grid: dims must be >= 1");
  const long long ncell = (long long)d->nx * d->ny * d->nz;
  if (ncell >= (1LL << 31)) return fail(RT_ERR_INVALID_ARG, "rt_create_grid: %lld cells exceed 2^31", ncell);
  if (!(d->box_len_cm > 0) || !isfinite(d->box_len_cm))
    return fail(RT_ERR_INVALID_ARG, "rt_create_grid: box_len_cm must be positive");
  if (d->precision != RT_FP64 && d->precision != RT_FP32_MIXED)
    return fail(RT_ERR_INVALID_ARG, "rt_create_grid: unknown precision %d", d->precision);
  if (d->mem_kind != RT_MEM_HOST && d->mem_kind != RT_MEM_DEVICE)
    return fail(RT_ERR_INVALID_ARG, "rt_create_grid: unknown mem_kind %d", d->mem_kind);
  if (!d->n_H || !d->x_HI) return fail(RT_ERR_INVALID_ARG, "rt_create_grid: n_H and x_HI are required");
  CUDA_TRY(cudaSetDevice(ctx->device));
  rt_grid* g = new rt_grid;
  g->ctx = ctx;
  g->nx = d->nx; g->ny = d->ny; g->nz = d->nz;
  g->ncell = ncell;
  g->box_len_cm = d->box_len_cm;
  g->dx = d->box_len_cm / d->nx;
  g->precision = d->precision;
  g->stream = (cudaStream_t)stream;
  const size_t n8 = (size_t)ncell * 8, ne = (size_t)ncell * elem_bytes(d->precision);
  int rc = RT_OK;
#define ALLOC(p, b)                                        \
  do {                                                     \
    cudaError_t e_ = cudaMalloc((void**)&(p), (b));        \
    if (e_ != cudaSuccess) {                               \
      delete g;                                            \
      return fail(RT_ERR_OOM, "rt_create_grid: cudaMalloc(%zu): %s", (size_t)(b), cudaGetErrorString(e_)); \
    }                                                      \
  } while (0)
  ALLOC(g->nH, n8);
  ALLOC(g->xHI, n8);
  ALLOC(g->xHII, n8);
  ALLOC(g->nhi, d->precision == RT_FP32_MIXED ? 2 * ne : ne);  // mixed: (hi, lo) pairs
  ALLOC(g->K, ne);
  ALLOC(g->G, ne);
  ALLOC(g->acc, kAccWords * sizeof(double));
  ALLOC(g->cnt, kCntWords * sizeof(unsigned long long));
  ALLOC(g->inst_dev, sizeof(InstDev));
  ALLOC(g->ts.ctl, CTL_N * sizeof(unsigned long long));
  ALLOC(g->ts.blk, blk_rows_bytes(ctx->num_sms, 1));
  g->ts.blk_blocks = ctx->num_sms * kBlkMaxPerSM;
  g->ts.blk_rows = 1;
#undef ALLOC
  cudaStream_t st = g->stream;
  if ((rc = upload(g->nH, d->n_H, n8, d->mem_kind, st)) != RT_OK) { delete g; return rc; }
  if ((rc = upload(g->xHI, d->x_HI, n8, d->mem_kind, st)) != RT_OK) { delete g; return rc; }
  // the values are checked on the device once they are there
  if ((rc = check_state("rt_create_grid", ncell, g->nH, g->xHI, st)) != RT_OK) { delete g; return rc; }
  if (d->x_HII) {
    if ((rc = upload(g->xHII, d->x_HII, n8, d->mem_kind, st)) != RT_OK) { delete g; return rc; }
  } else {
    cudaError_t e = launch_complement(ncell, g->xHI, g->xHII, st);
    if (e != cudaSuccess) { delete g; return fail(RT_ERR_CUDA, "complement: %s", cudaGetErrorString(e)); }
    g_launches.fetch_add(1);
  }
  cudaError_t e = launch_refresh(g->precision, ncell, g->nH, g->xHI, g->nhi, st);
  if (e != cudaSuccess) { delete g; return fail(RT_ERR_CUDA, "refresh: %s", cudaGetErrorString(e)); }
  g_launches.fetch_add(1);
  e = cudaMemsetAsync(g->ts.ctl, 0, CTL_N * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->K, 0, ne, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->G, 0, ne, st);
  const InstDev I = inst_of(g);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->inst_dev, &I, sizeof I, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMallocHost(&g->host_rb, 4096);
  if (e == cudaSuccess) e = cudaEventCreate(&g->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&g->ev1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { delete g; return fail(RT_ERR_CUDA, "rt_create_grid: %s", cudaGetErrorString(e)); }
  *out = g;
  g_last_error.clear();
  return RT_OK;
}

int rt_grid_destroy(rt_grid* g) {
  if (!g) return RT_OK;
  wait_batch(g);
  if (g->batch) detach_grid(g);
  cudaStreamSynchronize(g->stream);
  delete g;
  return RT_OK;
}

int rt_get_dims(rt_grid* g, int* nx, int* ny, int* nz) {
  if (!g || !nx || !ny || !nz) return fail(RT_ERR_INVALID_ARG, "rt_get_dims: NULL argument");
  *nx = g->nx;
  *ny = g->ny;
  *nz = g->nz;
  return RT_OK;
}

int rt_add_sources(rt_grid* g, int n, const double* pos, const double* ndot, const double* e_ph,
                   const double* sigma) {
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_add_sources: grid is NULL");
  if (n < 0) return fail(RT_ERR_INVALID_ARG, "rt_add_sources: n = %d", n);
  if (n == 0) return RT_OK;
  if (!pos || !ndot || !e_ph || !sigma) return fail(RT_ERR_INVALID_ARG, "rt_add_sources: NULL array");
  const double ext[3] = {g->nx * g->dx, g->ny * g->dx, g->nz * g->dx};
  for (int i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      const double p = pos[3 * i + a];
      if (!(p >= 0 && p <= ext[a])) return fail(RT_ERR_INVALID_ARG, "rt_add_sources: source %d axis %d at %g outside [0, %g]", i, a, p, ext[a]);
    }
    if (!(ndot[i] >= 0) || !isfinite(ndot[i])) return fail(RT_ERR_INVALID_ARG, "rt_add_sources: ndot[%d] = %g", i, ndot[i]);
    if (!(e_ph[i] >= kEHI) || !isfinite(e_ph[i])) return fail(RT_ERR_INVALID_ARG, "rt_add_sources: e_ph_eV[%d] = %g < 13.6", i, e_ph[i]);
    if (!(sigma[i] >= 0) || !isfinite(sigma[i])) return fail(RT_ERR_INVALID_ARG, "rt_add_sources: sigma[%d] = %g", i, sigma[i]);
  }
  if ((size_t)g->src_offset + g->src.size() + (size_t)n > (1u << 23))
    return fail(RT_ERR_INVALID_ARG, "rt_add_sources: too many sources");
  for (int i = 0; i < n; ++i) {
    rt_grid::SrcIn S;
    for (int a = 0; a < 3; ++a) S.pos[a] = pos[3 * i + a];
    S.ndot = ndot[i];
    S.e_ph = e_ph[i];
    S.sigma = sigma[i];
    g->src.push_back(S);
  }
  g->src_dirty = true;
  mark_batch_dirty(g);
  return RT_OK;
}

int rt_set_source_offset(rt_grid* g, int first) {
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_set_source_offset: grid is NULL");
  if (first < 0 || (size_t)first + g->src.size() > (1u << 23))
    return fail(RT_ERR_INVALID_ARG, "rt_set_source_offset: first = %d", first);
  g->src_offset = first;
  g->src_dirty = true;
  mark_batch_dirty(g);
  return RT_OK;
}

// Forget the packages in flight (finite speed of light).
static void drop_flight(rt_grid* g) {
  g->fl.live = false;
  g->fl.rlim.clear();
  g->fl.pend.clear();
  g->fl.unit.clear();
  g->fl.last_halted = 0;
}

int rt_clear_sources(rt_grid* g) {
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_clear_sources: grid is NULL");
  g->src.clear();
  g->src_dirty = true;
  mark_batch_dirty(g);
  drop_flight(g);
  return RT_OK;
}

int rt_set_source_rates(rt_grid* g, int n, const double* ndot) {
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_set_source_rates: grid is NULL");
  if (n != (int)g->src.size())
    return fail(RT_ERR_INVALID_ARG, "rt_set_source_rates: n = %d, the grid has %zu sources", n, g->src.size());
  if (n > 0 && !ndot) return fail(RT_ERR_INVALID_ARG, "rt_set_source_rates: ndot is NULL");
  for (int i = 0; i < n; ++i)
    if (!(ndot[i] >= 0) || !isfinite(ndot[i])) return fail(RT_ERR_INVALID_ARG, "rt_set_source_rates: ndot[%d] = %g", i, ndot[i]);
  for (int i = 0; i < n; ++i) g->src[i].ndot = ndot[i];
  g->src_dirty = true;
  mark_batch_dirty(g);
  return RT_OK;
}

// A source coordinate for which the FP32 walker may treat equal FP32 crossing
// distances of a 45-degree ray as an exact tie: a multiple of 1/16 no larger
// than 4096 cells, so every plane offset b - s is exact in FP32 and distinct
// offsets stay at least 1/16 apart.
static bool exact_in_f32(double v) { return v == ldexp(floor(ldexp(v, 4)), -4) && fabs(v) <= 4096.0; }

// Source records of grid g for a given initial level (Step 1: Ndot spread
// over 12 * 4^level0 root packages), attributed to instance slot `inst`.
// unit[i] / p0[i], when given, override the photons/s carried by P = 1 and
// the P of new packages (finite speed of light).
static void build_sources(const rt_grid* g, int level0, int inst, std::vector<SourceDev>& v,
                          const std::vector<double>* unit = nullptr, const std::vector<double>* p0 = nullptr) {
  const double npix0 = 12.0 * ldexp(1.0, 2 * level0);
  const double dx = g->dx, vol = dx * dx * dx;
  for (size_t i = 0; i < g->src.size(); ++i) {
    const rt_grid::SrcIn& H = g->src[i];
    SourceDev S;
    memset(&S, 0, sizeof S);
    for (int a = 0; a < 3; ++a) S.s[a] = H.pos[a] / dx;  // cell units
    S.sdx = H.sigma * dx;
    S.type = H.type;
    S.heat = (H.e_ph - kEIon[H.type]) * kEvErg;
    S.unit = unit ? (*unit)[i] : H.ndot / npix0;
    S.p0 = p0 ? (*p0)[i] : 1.0;
    S.w = S.unit * H.sigma / (dx * dx);
    S.rw = S.unit / vol;
    S.inst = inst;
    S.local = g->src_offset + (int)i;
    int exact = 1;
    float s32[3], slo[3], sab[3];
    for (int a = 0; a < 3; ++a) {
      s32[a] = (float)S.s[a];
      slo[a] = (float)(S.s[a] - (double)s32[a]);
      const bool pair_exact = (double)s32[a] + (double)slo[a] == S.s[a];
      sab[a] = pair_exact ? 0.0f : (float)(ldexp(fabs(S.s[a]), -46));
      exact &= exact_in_f32(S.s[a]) ? 1 : 0;
    }
    S.exact32 = exact && g->nx <= 4096 && g->ny <= 4096 && g->nz <= 4096;
    // the FP32 walker deposits Gamma in eV/s (rt_get_rates converts to erg/s)
    S.k32 = make_float4((float)S.sdx, (float)S.w, (float)S.rw, (float)(H.e_ph - kEIon[H.type]));
    S.s32 = make_float4(s32[0], s32[1], s32[2], S.exact32 ? 1.0f : 0.0f);
    S.slo32 = make_float4(slo[0], slo[1], slo[2], (float)(S.sdx - (double)(float)S.sdx));
    S.sabs32 = make_float4(sab[0], sab[1], sab[2], (float)S.p0);
    v.push_back(S);
  }
}

// Build the per-source device table of a single grid for a given initial
// level.  For a finite-speed-of-light trace, while packages are in flight a
// source keeps the unit their P values are expressed in, and its new
// packages carry P = (current rate / N_pix) / unit, so rate and level
// changes leave the packages in flight untouched.
static int prepare_sources(rt_grid* g, int level0, bool fsl) {
  if (!g->src_dirty && g->last_level0 == level0 && g->src_fsl == fsl) return RT_OK;
  std::vector<SourceDev> v;
  if (fsl) {
    const double npix0 = 12.0 * ldexp(1.0, 2 * level0);
    const size_t n = g->src.size();
    std::vector<double> unit(n), p0(n);
    for (size_t i = 0; i < n; ++i) {
      const double rate = g->src[i].ndot / npix0;
      const bool keep = g->fl.live && i < g->fl.unit.size() && g->fl.unit[i] > 0;
      unit[i] = keep ? g->fl.unit[i] : rate;
      p0[i] = unit[i] > 0 ? rate / unit[i] : 0.0;
    }
    g->fl.unit = unit;
    build_sources(g, level0, 0, v, &unit, &p0);
  } else {
    build_sources(g, level0, 0, v);
  }
  if (v.size() > g->src_dev_cap) {
    if (g->src_dev) cudaFree(g->src_dev);
    g->src_dev = nullptr;
    g->src_dev_cap = 0;
    const size_t cap = v.size() < 64 ? 64 : v.size();
    CUDA_TRY(cudaMalloc((void**)&g->src_dev, cap * sizeof(SourceDev)));
    g->src_dev_cap = cap;
  }
  if (!v.empty())
    CUDA_TRY(cudaMemcpyAsync(g->src_dev, v.data(), v.size() * sizeof(SourceDev), cudaMemcpyHostToDevice, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));  // v goes out of scope
  g->src_dirty = false;
  g->last_level0 = level0;
  g->src_fsl = fsl;
  return RT_OK;
}

static int check_params(const rt_trace_params* p) {
  if (!p) return fail(RT_ERR_INVALID_ARG, "rt_trace: params is NULL");
  if (p->level0 < 0 || p->level0 > RT_MAX_LEVEL) return fail(RT_ERR_INVALID_ARG, "rt_trace: level0 = %d", p->level0);
  if (p->max_level < p->level0 || p->max_level > RT_MAX_LEVEL)
    return fail(RT_ERR_INVALID_ARG, "rt_trace: max_level = %d", p->max_level);
  if (!(p->phi_c > 0) || !isfinite(p->phi_c)) return fail(RT_ERR_INVALID_ARG, "rt_trace: phi_c = %g", p->phi_c);
  if (!(p->f_term > 0 && p->f_term < 1)) return fail(RT_ERR_INVALID_ARG, "rt_trace: f_term = %g", p->f_term);
  if (p->queue_capacity < 0) return fail(RT_ERR_INVALID_ARG, "rt_trace: queue_capacity < 0");
  if (p->blocks_per_sm < 0 || p->blocks_per_sm > 32)
    return fail(RT_ERR_INVALID_ARG, "rt_trace: blocks_per_sm = %d", p->blocks_per_sm);
  if (p->segs_per_iter < 0 || p->segs_per_iter > 1024) return fail(RT_ERR_INVALID_ARG, "rt_trace: segs_per_iter = %d", p->segs_per_iter);
  if (p->passes < 0) return fail(RT_ERR_INVALID_ARG, "rt_trace: passes = %d", p->passes);
  if (!(p->light_cm >= 0) || !isfinite(p->light_cm)) return fail(RT_ERR_INVALID_ARG, "rt_trace: light_cm = %g", p->light_cm);
  return RT_OK;
}

// Queue of `cap` records of `rec` bytes (the layout of the next trace: a
// change of layout reallocates, which clears the tags).
static int ensure_queue(rt_grid* g, unsigned long long cap, size_t rec) {
  if (g->ts.queue && g->ts.cap >= cap && g->ts.rec_bytes == rec) return RT_OK;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (g->ts.queue) cudaFree(g->ts.queue);
  g->ts.queue = nullptr;
  g->ts.cap = 0;
  CUDA_TRY(cudaMalloc(&g->ts.queue, cap * rec));
  // tags start at 0; epochs start at 1
  CUDA_TRY(cudaMemsetAsync(g->ts.queue, 0, cap * rec, g->stream));
  g->ts.cap = cap;
  g->ts.rec_bytes = rec;
  return RT_OK;
}

static void fill_common_args(TraceArgs& A, const rt_trace_params* p) {
  for (int l = 0; l < kLevels; ++l) {
    // Eq. "split": Phi = N_pix dx^2 / (4 pi R^2) < Phi_c  <=>  R > R_split(l)
    A.rsplit[l] = sqrt((12.0 * ldexp(1.0, 2 * l)) / (4.0 * M_PI * p->phi_c));
    A.rsplit32[l] = (float)A.rsplit[l];
    A.rsplit32lo[l] = (float)(A.rsplit[l] - (double)A.rsplit32[l]);
  }
  A.level0 = p->level0;
  A.max_level = p->max_level;
  A.tau_term = -log(p->f_term);
  A.tau_term32 = (float)A.tau_term;
  A.tau_term32lo = (float)(A.tau_term - (double)A.tau_term32);
  A.timeout_ns = (long long)((p->timeout_s > 0 ? p->timeout_s : 2.0) * 1e9);
  A.segs_per_iter = p->segs_per_iter > 0 ? p->segs_per_iter : 8;
  A.checksums = (p->flags & RT_TRACE_CHECKSUMS) != 0;
  A.fc = (p->flags & RT_TRACE_FC) != 0;
  for (int l = 0; l < kLevels; ++l) {
    A.theta[l] = sqrt(4.0 * M_PI / (12.0 * ldexp(1.0, 2 * l)));
    A.theta32[l] = (float)A.theta[l];
  }
}

// One trace as `passes` launches of the trace kernel over consecutive, equal
// ranges of the sources, for traces whose packages do not fit the queue at
// once; deposits, budget sums and counters accumulate across the passes.
// A.npix0, A.queue, A.cap, A.ctl and the per-trace fields are set by the
// caller; A.src, A.nsrc, A.src_first and A.n_roots are set here per pass.  Packages in
// flight (fsl) are shared out over the passes on the device; `mode` and
// `in_cap` say what the first pass takes over from the previous trace.
static int launch_passes(TraceArgs A, size_t queue_bytes, const SourceDev* src, int nsrc, int passes, int precision,
                         int fsl, int mode, unsigned long long in_cap, int blocks, cudaEvent_t ev0, cudaEvent_t ev1,
                         cudaStream_t st, bool stall = false) {
  if ((unsigned long long)nsrc >= kMaxQueueSources)
    return fail(RT_ERR_INVALID_ARG, "trace: %d sources in one launch (at most %u)", nsrc, kMaxQueueSources - 1u);
  if (passes > nsrc) passes = nsrc;
  if (passes < 1) passes = 1;
  for (int i = 0; i < passes; ++i) {
    const int s0 = (int)((long long)nsrc * i / passes);
    const int s1 = (int)((long long)nsrc * (i + 1) / passes);
    const unsigned long long n = (unsigned long long)A.npix0 * (unsigned long long)(s1 - s0);
    LAUNCH_TRY(launch_trace_init(A.ctl, A.queue, queue_bytes, n, i == 0, mode, in_cap, i, passes, st));
    // self-test: one package that never exists keeps the trace from ending,
    // so its bounded waits must run out (RT_TRACE_SELFTEST_STALL)
    if (i == 0 && stall) LAUNCH_TRY(launch_add_word(A.ctl + CTL_OUTSTANDING, 1ULL, st));
    if (i == 0) CUDA_TRY(cudaEventRecord(ev0, st));
    if (n == 0 && !fsl) continue;
    A.src = src;
    A.nsrc = nsrc;
    A.src_first = s0;
    A.n_roots = n;
    LAUNCH_TRY(launch_trace(precision, fsl, A, blocks, 256, st));
  }
  CUDA_TRY(cudaEventRecord(ev1, st));
  return RT_OK;
}

// Largest automatically sized queue: 2^31 records, and at most half of the
// device memory that is free (counting the queue it would replace).
static unsigned long long queue_cap_limit(size_t rec, size_t held_bytes) {
  unsigned long long lim = 1ULL << 31;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
    const unsigned long long m = ((unsigned long long)fr + held_bytes) / 2 / rec;
    if (m < lim) lim = m;
  } else {
    cudaGetLastError();
  }
  if (lim < (1ULL << 20)) lim = 1ULL << 20;
  return lim;
}


// Device buffer of at least `bytes`, reallocated (after the stream's work
// is done) when smaller.
static int ensure_buffer(void** p, size_t* have, size_t bytes, cudaStream_t st) {
  if (*p && *have >= bytes) return RT_OK;
  CUDA_TRY(cudaStreamSynchronize(st));
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  CUDA_TRY(cudaMalloc(p, bytes));
  *have = bytes;
  return RT_OK;
}

constexpr unsigned long long kFlightMinCap = 1ULL << 16;  // records of a new in-flight store
constexpr size_t kFlightMaxAges = 1u << 20;

// Finite speed of light, before the launches of a trace: the halting radii of
// this trace (advanced from the last trace's on the device; on a retry of
// the same trace they stand) and room for the packages it halts.
static int prepare_flight(rt_grid* g, const rt_trace_params* p, bool retry, TraceArgs& A) {
  FlightState& F = g->fl;
  cudaStream_t st = g->stream;
  const double c_dt = p->light_cm / g->dx;  // cell units
  if (!retry) {
    const double diag = sqrt((double)g->nx * g->nx + (double)g->ny * g->ny + (double)g->nz * g->nz);
    std::vector<double> neu;
    flight_radii(F.rlim, F.live, c_dt, diag, neu);
    const size_t n_new = neu.size();
    if (n_new > kFlightMaxAges)
      return fail(RT_ERR_INVALID_ARG, "rt_trace: light_cm = %g cm is too short for this grid (%zu ages in flight)",
                  p->light_cm, n_new);
    const int nt = 1 - F.tab;
    size_t have64 = F.rlim_cap[nt] * sizeof(double), have32 = F.rlim_cap[nt] * sizeof(float2);
    if (F.rlim_cap[nt] < n_new) {
      const size_t cap = n_new < 64 ? 64 : 2 * n_new;
      have64 = have32 = 0;
      F.rlim_cap[nt] = 0;  // the old tables are released even if the new ones cannot be had
      int rc = ensure_buffer((void**)&F.rlim64[nt], &have64, cap * sizeof(double), st);
      if (!rc) rc = ensure_buffer((void**)&F.rlim32[nt], &have32, cap * sizeof(float2), st);
      if (rc) return rc;
      F.rlim_cap[nt] = cap;
    }
    LAUNCH_TRY(launch_flight_table(F.rlim64[F.tab], F.rlim64[nt], F.rlim32[nt], (int)n_new, c_dt, st));
    F.pend.swap(neu);  // the launch adopts them (commit_flight); a failed one leaves rlim as it was
  }
  const int tab = retry ? F.tab : 1 - F.tab;
  const size_t n_ages = retry ? F.rlim.size() : F.pend.size();
  // the output store: the other buffer than the one holding the last trace's packages
  const int out = F.live ? 1 - F.in : F.in;
  unsigned long long want = F.last_halted + F.last_halted / 4 + 1024;
  if (want < kFlightMinCap) want = kFlightMinCap;
  if (F.cap[out] < want) {
    const size_t rec = g->precision == RT_FP64 ? sizeof(Rec64) : sizeof(Rec32);
    size_t have = 0;
    F.cap[out] = 0;  // the old store is released even if the new one cannot be had
    int rc = ensure_buffer(&F.buf[out], &have, want * rec, st);
    if (rc) return rc;
    F.cap[out] = want;
  }
  A.rlim64 = F.rlim64[tab];
  A.rlim32 = F.rlim32[tab];
  A.n_ages = (int)n_ages;
  A.res_in = F.live ? F.buf[F.in] : nullptr;
  A.halt_out = F.buf[out];
  A.halt_cap = F.cap[out];
  return RT_OK;
}


static void commit_flight(rt_grid* g, bool fsl);

static int enqueue_trace(rt_grid* g, const rt_trace_params* p, int passes, bool retry = false) {
  const bool fsl = p->light_cm > 0;
  for (const rt_grid::SrcIn& S : g->src)
    if (S.type > 0 && !g->he)
      return fail(RT_ERR_INVALID_ARG, "rt_trace: helium photon types need rt_set_absorbers first");
  if (retry) {
    g->fl.in = g->fl.in_before;
    g->fl.live = g->fl.live_before;
  } else {
    g->fl.in_before = g->fl.in;
    g->fl.live_before = g->fl.live;
  }
  int rc = prepare_sources(g, p->level0, fsl);
  if (rc) return rc;
  cudaStream_t st = g->stream;
  const size_t ne = (size_t)g->ncell * elem_bytes(g->precision);
  // Step 2: k_ph, Gamma and the budget words in one launch
  LAUNCH_TRY(launch_zero_fields(g->K, g->G, ne, g->acc, kAccWords, g->cnt, kCntWords, st));
  for (int t = 0; t < 2 && g->he; ++t) {
    CUDA_TRY(cudaMemsetAsync(g->Khe[t], 0, ne, st));
    CUDA_TRY(cudaMemsetAsync(g->Ghe[t], 0, ne, st));
  }
  const int nsrc = (int)g->src.size();
  if (nsrc == 0) {
    LAUNCH_TRY(launch_trace_init(g->ts.ctl, g->ts.queue, g->ts.cap * g->ts.rec_bytes, 0, 1, FLIGHT_OFF, 0, 0, 1, st));
    drop_flight(g);
    g->traced = false;
    g->ts.passes_run = 0;
    return RT_OK;
  }
  TraceArgs A;
  memset(&A, 0, sizeof A);
  fill_common_args(A, p);
  A.inst = g->inst_dev;
  A.ninst = 1;
  A.npix0 = (uint32_t)(12u << (2 * p->level0));
  A.dir_tab = nullptr;
  A.dir_levels = -1;
  if (g->precision == RT_FP32_MIXED) {
    // deepest level a package can reach: R_split(l) >= box diagonal stops splitting
    const double diag = sqrt((double)g->nx * g->nx + (double)g->ny * g->ny + (double)g->nz * g->nz);
    int need = p->level0;
    while (need < p->max_level && A.rsplit[need] < diag) ++need;
    const int want = need < kDirTableMaxLevel ? need : kDirTableMaxLevel;
    int rc2 = ensure_dir_table(g->ctx, want, &A.dir_tab, &A.dir_levels);
    if (rc2) return rc2;
  }
  A.queue = g->ts.queue;
  A.cap = g->ts.cap;
  A.ctl = g->ts.ctl;
  A.max_steps = 2 * (g->nx + g->ny + g->nz) + 16;
  if (p->segs_per_iter == 0) A.segs_per_iter = tuned_segs_per_iter(g->seg_per_pkg, !fsl);
  int mode = FLIGHT_OFF;
  unsigned long long in_cap = 0;
  if (fsl) {
    if ((rc = prepare_flight(g, p, retry, A))) return rc;
    mode = retry ? FLIGHT_RETRY : (g->fl.live ? FLIGHT_ADVANCE : FLIGHT_OFF);
    in_cap = g->fl.live ? g->fl.cap[g->fl.in] : 0;
  }
  const int block = 256;  // the trace kernel is compiled for 256-thread blocks
  int per_sm = 0;
  CUDA_TRY(trace_occupancy(g->precision, fsl ? 1 : 0, block, &per_sm));
  if (per_sm < 1) per_sm = 1;
  if (p->blocks_per_sm > 0 && p->blocks_per_sm < per_sm) per_sm = p->blocks_per_sm;
  if ((rc = g->ts.bind_rows(A, per_sm * g->ctx->num_sms, 1))) return rc;
  if ((rc = launch_passes(A, g->ts.cap * g->ts.rec_bytes, g->src_dev, nsrc, passes, g->precision, fsl ? 1 : 0, mode,
                          in_cap, per_sm * g->ctx->num_sms, g->ev0, g->ev1, st, (p->flags & RT_TRACE_SELFTEST_STALL) != 0)))
    return rc;
  commit_flight(g, fsl);
  g->traced = true;
  g->ts.passes_run = passes < nsrc ? passes : nsrc;
  return RT_OK;
}

// After the launches of a trace: with a finite speed of light its output
// store now holds the packages in flight and its halting radii are the
// current ones; otherwise nothing is in flight.
static void commit_flight(rt_grid* g, bool fsl) {
  FlightState& F = g->fl;
  if (!fsl) {
    drop_flight(g);
    return;
  }
  if (!F.pend.empty()) {
    F.tab = 1 - F.tab;
    F.rlim.swap(F.pend);
    F.pend.clear();
  }
  if (F.live) F.in = 1 - F.in;
  F.live = true;
}

// A state uploaded by rt_set_state_async failed its check on the device:
// keep the message for the caller and clear the device's latch (the grid kept
// its previous state).
static void note_rejected_state(rt_grid* g, unsigned long long bad_n, unsigned long long bad_x) {
  char buf[160];
  if (bad_n != ~0ULL)
    snprintf(buf, sizeof buf, "rt_set_state_async: n_H[%llu] is negative or not finite; the state was not changed",
             bad_n);
  else
    snprintf(buf, sizeof buf, "rt_set_state_async: x_HI[%llu] lies outside [0, 1]; the state was not changed", bad_x);
  g->set_err = buf;
  cudaMemsetAsync(g->ts.ctl + CTL_SET_ERR, 0, sizeof(unsigned long long), g->stream);
}

static int read_budget(rt_grid* g, rt_budget* out) {
  double* hacc = (double*)g->host_rb;
  unsigned long long* hcnt = (unsigned long long*)((char*)g->host_rb + 64);
  unsigned long long* hctl = (unsigned long long*)((char*)g->host_rb + 512);
  cudaStream_t st = g->stream;
  CUDA_TRY(cudaMemcpyAsync(hacc, g->acc, kAccWords * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(hcnt, g->cnt, kCntWords * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(hctl, g->ts.ctl, CTL_N * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  memset(out, 0, sizeof *out);
  out->emitted = hacc[0];
  out->absorbed = hacc[1];
  out->escaped = hacc[2];
  for (int l = 0; l < kLevels; ++l) {
    out->counts[l] = hcnt[l];
    out->hashes[l] = hcnt[kLevels + l];
  }
  out->segments = hcnt[kCntSegments];
  out->fallbacks = hcnt[kCntFallbacks];
  out->fallbacks_tau = hcnt[kCntFallbacksTau];
  out->queue_pushed = hctl[CTL_PUSHED] + hctl[CTL_TAIL];
  out->queue_peak = hctl[CTL_PEAK] > hctl[CTL_TAIL] ? hctl[CTL_PEAK] : hctl[CTL_TAIL];
  out->passes = g->ts.passes_run;
  out->status = (int)hctl[CTL_STATUS];
  out->resumed = hacc[3];
  out->halted = hacc[4];
  out->n_resumed = hctl[CTL_RESUME];
  out->n_halted = hctl[CTL_HALTED];
  if (hctl[CTL_SET_ERR]) {
    note_rejected_state(g, hctl[CTL_SET_BADN], hctl[CTL_SET_BADX]);
    out->status = RT_ERR_INVALID_ARG;
  }
  if (g->fl.live) g->fl.last_halted = out->n_halted;
  unsigned long long pkgs = out->n_resumed;
  for (int l = 0; l < kLevels; ++l) pkgs += out->counts[l];
  if (out->status == RT_OK && pkgs > 0) g->seg_per_pkg = (double)out->segments / (double)pkgs;
  float ms = 0.f;
  if (g->traced && cudaEventElapsedTime(&ms, g->ev0, g->ev1) == cudaSuccess) out->kernel_ms = ms;
  else cudaGetLastError();
  return RT_OK;
}

int rt_trace(rt_grid* g, const rt_trace_params* p, rt_budget* out) {
  NvtxRange nr("rt_trace");
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_trace: grid is NULL");
  if (int rcw = wait_batch(g)) return rcw;
  int rc = check_params(p);
  if (rc) return rc;
  CUDA_TRY(cudaSetDevice(g->ctx->device));
  unsigned long long cap = (unsigned long long)p->queue_capacity;
  const bool automatic = cap == 0;
  if (automatic) {
    cap = g->ts.cap;
    if (cap == 0) {
      cap = (unsigned long long)g->ncell * 4ULL;
      if (cap < (1ULL << 20)) cap = 1ULL << 20;
      if (cap > (1ULL << 26)) cap = 1ULL << 26;
    }
  }
  const bool fsl = p->light_cm > 0;
  const size_t rec = queue_rec_bytes(g->precision == RT_FP64, fsl);
  const int p_min = p->passes > 1 ? p->passes : 1;
  int passes = automatic && g->ts.passes > p_min ? g->ts.passes : p_min;
  const int nsrc = (int)g->src.size();
  for (int attempt = 0;; ++attempt) {
    if ((rc = ensure_queue(g, cap, rec))) return rc;
    if ((rc = enqueue_trace(g, p, passes, attempt > 0))) return rc;
    if (!out) return RT_OK;
    if ((rc = read_budget(g, out))) return rc;
    if (out->status == RT_ERR_QUEUE_OVERFLOW && attempt < 40) {
      // the store of halted packages grows by itself (read_budget noted how
      // many there were); the queue when it is sized automatically
      bool again = fsl && out->n_halted > g->fl.cap[g->fl.in];
      if (out->queue_peak > g->ts.cap) {
        const unsigned long long limit = queue_cap_limit(rec, (size_t)g->ts.cap * g->ts.rec_bytes);
        again = automatic && grow_after_overflow(out->queue_peak, limit, nsrc, &cap, &passes);
      }
      if (again) continue;
    }
    if (out->status == RT_ERR_INVALID_ARG && !g->set_err.empty())
      return fail(RT_ERR_INVALID_ARG, "rt_trace: %s", g->set_err.c_str());
    if (out->status != RT_OK)
      return fail(out->status, "rt_trace: device status %d (queue capacity %llu, largest pass %llu, passes %d)",
                  out->status, (unsigned long long)g->ts.cap, (unsigned long long)out->queue_peak, out->passes);
    if (automatic) {
      // remember the passes the sizing added (halved while the queue is
      // under a quarter full), not the caller's minimum
      if (passes > p_min) g->ts.passes = 4 * out->queue_peak < g->ts.cap ? passes / 2 : passes;
      // a repeat of this trace may send every child that is not child 0
      // through the queue (which of them a free lane of the splitting warp
      // takes depends on scheduling): keep room for that
      if (out->passes <= 1) {
        const unsigned long long need = queue_worst_case(out->counts, p->level0, kLevels);
        if (need > g->ts.cap) {
          const unsigned long long limit = queue_cap_limit(rec, (size_t)g->ts.cap * g->ts.rec_bytes);
          const unsigned long long want = need + need / 8 + 1024;
          if (want <= limit && (rc = ensure_queue(g, want, rec))) return rc;
        }
      }
    }
    return RT_OK;
  }
}

int rt_get_budget(rt_grid* g, rt_budget* out) {
  if (!g || !out) return fail(RT_ERR_INVALID_ARG, "rt_get_budget: NULL argument");
  if (int rcw = wait_batch(g)) return rcw;
  int rc = read_budget(g, out);
  if (rc) return rc;
  if (out->status == RT_ERR_INVALID_ARG && !g->set_err.empty())
    return fail(RT_ERR_INVALID_ARG, "rt_get_budget: %s", g->set_err.c_str());
  if (out->status != RT_OK) return fail(out->status, "rt_get_budget: device status %d", out->status);
  return RT_OK;
}

int rt_chem_update(rt_grid* g, double dt_s, int nsub, double alpha_B) {
  NvtxRange nr("rt_chem_update");
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_chem_update: grid is NULL");
  if (int rcw = wait_batch(g)) return rcw;
  if (!(dt_s >= 0) || !isfinite(dt_s)) return fail(RT_ERR_INVALID_ARG, "rt_chem_update: dt_s = %g", dt_s);
  if (nsub < 1) return fail(RT_ERR_INVALID_ARG, "rt_chem_update: nsub = %d", nsub);
  if (!(alpha_B >= 0) || !isfinite(alpha_B)) return fail(RT_ERR_INVALID_ARG, "rt_chem_update: alpha_B = %g", alpha_B);
  CUDA_TRY(cudaSetDevice(g->ctx->device));
  const double h = dt_s / nsub;
  LAUNCH_TRY(launch_chem(g->precision, g->ncell, g->nH, g->xHI, g->xHII, g->K, g->nhi, h, nsub, alpha_B, g->stream));
  return RT_OK;
}

int rt_set_state(rt_grid* g, const double* n_H, const double* x_HI, const double* x_HII, int mem_kind) {
  NvtxRange nr("rt_set_state");
  if (!g || !x_HI) return fail(RT_ERR_INVALID_ARG, "rt_set_state: grid and x_HI are required");
  if (int rcw = wait_batch(g)) return rcw;
  if (mem_kind != RT_MEM_HOST && mem_kind != RT_MEM_DEVICE) return fail(RT_ERR_INVALID_ARG, "rt_set_state: mem_kind %d", mem_kind);
  CUDA_TRY(cudaSetDevice(g->ctx->device));
  const long long ncell = g->ncell;
  const size_t n8 = (size_t)ncell * 8;
  cudaStream_t st = g->stream;
  // stage the new state on the device, check it there, and only then replace
  // the grid's state (which an invalid call leaves unchanged)
  const int nf = (n_H ? 1 : 0) + 1 + (x_HII ? 1 : 0);
  double* stage = nullptr;
  CUDA_TRY(cudaMallocAsync((void**)&stage, nf * n8, st));
  double* sn = n_H ? stage : nullptr;
  double* sx = stage + (n_H ? ncell : 0);
  double* sz = x_HII ? sx + ncell : nullptr;
  int rc = RT_OK;
  if (n_H) rc = upload(sn, n_H, n8, mem_kind, st);
  if (!rc) rc = upload(sx, x_HI, n8, mem_kind, st);
  if (!rc && x_HII) rc = upload(sz, x_HII, n8, mem_kind, st);
  if (!rc) rc = check_state("rt_set_state", ncell, sn, sx, st);
  if (rc) {
    cudaFreeAsync(stage, st);
    return rc;
  }
  if (n_H) CUDA_TRY(cudaMemcpyAsync(g->nH, sn, n8, cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(g->xHI, sx, n8, cudaMemcpyDeviceToDevice, st));
  if (x_HII) {
    CUDA_TRY(cudaMemcpyAsync(g->xHII, sz, n8, cudaMemcpyDeviceToDevice, st));
  } else {
    LAUNCH_TRY(launch_complement(ncell, g->xHI, g->xHII, st));
  }
  LAUNCH_TRY(launch_refresh(g->precision, ncell, g->nH, g->xHI, g->nhi, st));
  CUDA_TRY(cudaFreeAsync(stage, st));
  return RT_OK;
}

// The FP32-mixed grid keeps Gamma in eV/s (FP32 erg/s values of faint cells
// fall below the FP32 normal range); this scale turns it into erg/s.
static double gamma_scale(const rt_grid* g) { return g->precision == RT_FP64 ? 1.0 : kEvErg; }

// Streams, events and (when `stage_up` / `stage_dn`) staging areas of the
// calls that do not wait.  Allocating synchronises the device: the first
// such call on a grid does it.
static int ensure_async(rt_grid* g, bool stage_up, bool stage_dn) {
  if (!g->up) CUDA_TRY(cudaStreamCreateWithFlags(&g->up, cudaStreamNonBlocking));
  if (!g->dn) CUDA_TRY(cudaStreamCreateWithFlags(&g->dn, cudaStreamNonBlocking));
  cudaEvent_t* evs[6] = {&g->ev_up, &g->ev_commit, &g->ev_snap, &g->ev_dl[0], &g->ev_dl[1], &g->ev_dl[2]};
  for (cudaEvent_t* ev : evs)
    if (!*ev) CUDA_TRY(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
  const size_t n8 = (size_t)g->ncell * 8;
  if (stage_up && !g->up_stage) CUDA_TRY(cudaMalloc((void**)&g->up_stage, 3 * n8));  // uploads with n_H
  if (stage_dn && !g->dn_stage) CUDA_TRY(cudaMalloc((void**)&g->dn_stage, 3 * n8));
  if (!g->check_words_set) {
    // ~0 = no failing cell; every commit leaves them so for the next upload
    CUDA_TRY(cudaMemsetAsync(g->ts.ctl + CTL_CHECK_N, 0xff, 2 * sizeof(unsigned long long), g->stream));
    g->check_words_set = true;
  }
  return RT_OK;
}

int rt_set_state_async(rt_grid* g, const double* n_H, const double* x_HI, const double* x_HII, int mem_kind) {
  NvtxRange nr("rt_set_state_async");
  if (!g || !x_HI) return fail(RT_ERR_INVALID_ARG, "rt_set_state_async: grid and x_HI are required");
  if (mem_kind != RT_MEM_HOST && mem_kind != RT_MEM_DEVICE)
    return fail(RT_ERR_INVALID_ARG, "rt_set_state_async: mem_kind %d", mem_kind);
  if (g->batch) return fail(RT_ERR_STATE, "rt_set_state_async: the grid is in a batch (use rt_set_state)");
  CUDA_TRY(cudaSetDevice(g->ctx->device));
  int rc = ensure_async(g, mem_kind == RT_MEM_HOST && n_H != nullptr, false);
  if (rc) return rc;
  const long long n = g->ncell;
  const size_t n8 = (size_t)n * 8;
  cudaStream_t st = g->stream;
  const double* sn = n_H;
  const double* sx = x_HI;
  const double* sz = x_HII;
  if (mem_kind == RT_MEM_HOST && !n_H) {
    // Straight into the alternate buffers, which the grid's kernels last
    // used before the previous commit; one kernel checks the new state and
    // refreshes n_HI (undoing it if rejected), and the buffers swap.
    if (!g->xHI_alt) CUDA_TRY(cudaMalloc((void**)&g->xHI_alt, n8));
    if (!g->xHII_alt) CUDA_TRY(cudaMalloc((void**)&g->xHII_alt, n8));
    CUDA_TRY(cudaStreamWaitEvent(g->up, g->ev_commit, 0));
    CUDA_TRY(cudaMemcpyAsync(g->xHI_alt, x_HI, n8, cudaMemcpyHostToDevice, g->up));
    if (x_HII) CUDA_TRY(cudaMemcpyAsync(g->xHII_alt, x_HII, n8, cudaMemcpyHostToDevice, g->up));
    CUDA_TRY(cudaEventRecord(g->ev_up, g->up));
    CUDA_TRY(cudaStreamWaitEvent(st, g->ev_up, 0));
    LAUNCH_TRY(launch_check_refresh(g->precision, n, g->ts.ctl, g->nH, g->xHI_alt, g->xHII_alt, x_HII != nullptr,
                                    g->xHI, g->xHII, g->nhi, g->inst_dev, st));
    CUDA_TRY(cudaEventRecord(g->ev_commit, st));
    std::swap(g->xHI, g->xHI_alt);
    std::swap(g->xHII, g->xHII_alt);
    return RT_OK;
  }
  if (mem_kind == RT_MEM_HOST) {
    // the staging area is free once the previous commit has read it
    CUDA_TRY(cudaStreamWaitEvent(g->up, g->ev_commit, 0));
    double* d = g->up_stage;
    if (n_H) CUDA_TRY(cudaMemcpyAsync(d, n_H, n8, cudaMemcpyHostToDevice, g->up));
    CUDA_TRY(cudaMemcpyAsync(d + n, x_HI, n8, cudaMemcpyHostToDevice, g->up));
    if (x_HII) CUDA_TRY(cudaMemcpyAsync(d + 2 * n, x_HII, n8, cudaMemcpyHostToDevice, g->up));
    CUDA_TRY(cudaEventRecord(g->ev_up, g->up));
    CUDA_TRY(cudaStreamWaitEvent(st, g->ev_up, 0));
    sn = n_H ? d : nullptr;
    sx = d + n;
    sz = x_HII ? d + 2 * n : nullptr;
  }
  LAUNCH_TRY(launch_check_state(n, sn, sx, g->ts.ctl + CTL_CHECK_N, st));
  LAUNCH_TRY(launch_commit_state(g->precision, n, g->ts.ctl, sn, sx, sz, g->nH, g->xHI, g->xHII, g->nhi, st));
  CUDA_TRY(cudaEventRecord(g->ev_commit, st));
  return RT_OK;
}

// One field into a snapshot or a caller's device buffer: a device-to-device
// copy when neither the element type nor the scale changes, else the
// conversion kernel.
static int copy_or_convert(long long n, const void* src, int sdt, void* dst, int ddt, double scale, cudaStream_t st) {
  if (sdt == ddt && scale == 1.0) {
    CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)n * (sdt == RT_DTYPE_F64 ? 8 : 4), cudaMemcpyDeviceToDevice, st));
    return RT_OK;
  }
  LAUNCH_TRY(launch_convert(n, src, sdt, dst, ddt, st, scale));
  return RT_OK;
}

int rt_get_rates_async(rt_grid* g, void* kph, void* gamma, void* x_HI, int dtype, int mem_kind) {
  NvtxRange nr("rt_get_rates_async");
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_get_rates_async: grid is NULL");
  if (dtype != RT_DTYPE_F64 && dtype != RT_DTYPE_F32)
    return fail(RT_ERR_INVALID_ARG, "rt_get_rates_async: dtype %d", dtype);
  if (mem_kind != RT_MEM_HOST && mem_kind != RT_MEM_DEVICE)
    return fail(RT_ERR_INVALID_ARG, "rt_get_rates_async: mem_kind %d", mem_kind);
  if (g->batch) return fail(RT_ERR_STATE, "rt_get_rates_async: the grid is in a batch (use rt_get_rates)");
  CUDA_TRY(cudaSetDevice(g->ctx->device));
  const int kd = g->precision == RT_FP64 ? RT_DTYPE_F64 : RT_DTYPE_F32;
  const void* src[3] = {g->K, g->G, g->xHI};
  const int sdt[3] = {kd, kd, RT_DTYPE_F64};
  const double scale[3] = {1.0, gamma_scale(g), 1.0};
  void* dst[3] = {kph, gamma, x_HI};
  const long long n = g->ncell;
  cudaStream_t st = g->stream;
  if (mem_kind == RT_MEM_DEVICE) {
    for (int f = 0; f < 3; ++f)
      if (dst[f]) {
        int rc = copy_or_convert(n, src[f], sdt[f], dst[f], dtype, scale[f], st);
        if (rc) return rc;
      }
    return RT_OK;
  }
  int rc = ensure_async(g, false, true);
  if (rc) return rc;
  const size_t eb = dtype == RT_DTYPE_F64 ? 8 : 4, region = (size_t)n * 8;
  // a field's staging region is free once its previous read-back has left it
  for (int f = 0; f < 3; ++f) {
    if (!dst[f]) continue;
    CUDA_TRY(cudaStreamWaitEvent(st, g->ev_dl[f], 0));
    if ((rc = copy_or_convert(n, src[f], sdt[f], g->dn_stage + f * region, dtype, scale[f], st))) return rc;
  }
  CUDA_TRY(cudaEventRecord(g->ev_snap, st));
  CUDA_TRY(cudaStreamWaitEvent(g->dn, g->ev_snap, 0));
  for (int f = 0; f < 3; ++f) {
    if (!dst[f]) continue;
    CUDA_TRY(cudaMemcpyAsync(dst[f], g->dn_stage + f * region, (size_t)n * eb, cudaMemcpyDeviceToHost, g->dn));
    CUDA_TRY(cudaEventRecord(g->ev_dl[f], g->dn));
  }
  return RT_OK;
}

int rt_wait_rates(rt_grid* g) {
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_wait_rates: grid is NULL");
  for (int f = 0; f < 3; ++f)
    if (g->ev_dl[f]) CUDA_TRY(cudaEventSynchronize(g->ev_dl[f]));
  return RT_OK;
}

static int copy_field(rt_grid* g, const void* src, int src_dtype, void* dst, int dtype, int mem_kind,
                      double scale = 1.0) {
  if (!dst) return RT_OK;
  const long long n = g->ncell;
  const size_t eb = dtype == RT_DTYPE_F64 ? 8 : 4;
  cudaStream_t st = g->stream;
  if (mem_kind == RT_MEM_DEVICE) {
    LAUNCH_TRY(launch_convert(n, src, src_dtype, dst, dtype, st, scale));
    return RT_OK;
  }
  if (src_dtype == dtype && scale == 1.0) {  // same type: straight to the host
    CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)n * eb, cudaMemcpyDeviceToHost, st));
    return RT_OK;
  }
  void* tmp = nullptr;
  CUDA_TRY(cudaMallocAsync(&tmp, (size_t)n * eb, st));
  cudaError_t e = launch_convert(n, src, src_dtype, tmp, dtype, st, scale);
  if (e == cudaSuccess) {
    g_launches.fetch_add(1);
    e = cudaMemcpyAsync(dst, tmp, (size_t)n * eb, cudaMemcpyDeviceToHost, st);
  }
  cudaFreeAsync(tmp, st);
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, "copy_field: %s", cudaGetErrorString(e));
  return RT_OK;
}

int rt_set_absorbers(rt_grid* g, const double* n_HeI, const double* n_HeII, int mem_kind) {
  if (!g || !n_HeI || !n_HeII) return fail(RT_ERR_INVALID_ARG, "rt_set_absorbers: NULL argument");
  if (int rcw = wait_batch(g)) return rcw;
  if (mem_kind != RT_MEM_HOST && mem_kind != RT_MEM_DEVICE)
    return fail(RT_ERR_INVALID_ARG, "rt_set_absorbers: mem_kind %d", mem_kind);
  CUDA_TRY(cudaSetDevice(g->ctx->device));
  cudaStream_t st = g->stream;
  const long long n = g->ncell;
  const size_t n8 = (size_t)n * 8, ne = (size_t)n * elem_bytes(g->precision);
  // staged and checked before the grid's arrays change
  double* stage = nullptr;
  CUDA_TRY(cudaMallocAsync((void**)&stage, 2 * n8, st));
  unsigned long long* bad = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&bad, 2 * sizeof(unsigned long long), st);
  unsigned long long h[2] = {~0ULL, ~0ULL};
  const cudaMemcpyKind kind = mem_kind == RT_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage, n_HeI, n8, kind, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage + n, n_HeII, n8, kind, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0xff, 2 * sizeof(unsigned long long), st);
  for (int t = 0; t < 2 && e == cudaSuccess; ++t) {
    e = launch_check_density(n, stage + t * n, bad + t, st);
    if (e == cudaSuccess) g_launches.fetch_add(1);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, bad, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(bad, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(stage, st);
    return fail(RT_ERR_CUDA, "rt_set_absorbers: %s", cudaGetErrorString(e));
  }
  for (int t = 0; t < 2; ++t) {
    if (h[t] == ~0ULL) continue;
    cudaFreeAsync(stage, st);
    return fail(RT_ERR_INVALID_ARG, "rt_set_absorbers: %s[%llu] is negative or not finite", t ? "n_HeII" : "n_HeI", h[t]);
  }
  if (!g->he) {
    for (int t = 0; t < 2; ++t) {
      e = cudaMalloc((void**)&g->nhe64[t], n8);
      if (e == cudaSuccess) {
        if (g->precision == RT_FP64) g->nhe[t] = g->nhe64[t];
        else e = cudaMalloc(&g->nhe[t], 2 * ne);  // FP32 pairs
      }
      if (e == cudaSuccess) e = cudaMalloc(&g->Khe[t], ne);
      if (e == cudaSuccess) e = cudaMalloc(&g->Ghe[t], ne);
      if (e == cudaSuccess) e = cudaMemsetAsync(g->Khe[t], 0, ne, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(g->Ghe[t], 0, ne, st);
      if (e != cudaSuccess) {
        cudaFreeAsync(stage, st);
        cudaStreamSynchronize(st);
        for (int u = 0; u < 2; ++u) {  // leave the grid as it was
          if (g->nhe[u] != g->nhe64[u]) cudaFree(g->nhe[u]);
          cudaFree(g->nhe64[u]); cudaFree(g->Khe[u]); cudaFree(g->Ghe[u]);
          g->nhe[u] = g->Khe[u] = g->Ghe[u] = nullptr;
          g->nhe64[u] = nullptr;
        }
        return fail(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "rt_set_absorbers: %s",
                    cudaGetErrorString(e));
      }
    }
    g->he = true;
    const InstDev I = inst_of(g);
    CUDA_TRY(cudaMemcpyAsync(g->inst_dev, &I, sizeof I, cudaMemcpyHostToDevice, st));
  }
  for (int t = 0; t < 2; ++t) {
    CUDA_TRY(cudaMemcpyAsync(g->nhe64[t], stage + t * n, n8, cudaMemcpyDeviceToDevice, st));
    if (g->precision == RT_FP32_MIXED) LAUNCH_TRY(launch_pair(n, g->nhe64[t], g->nhe[t], st));
  }
  cudaFreeAsync(stage, st);
  CUDA_TRY(cudaStreamSynchronize(st));
  mark_batch_dirty(g);
  return RT_OK;
}

int rt_set_source_types(rt_grid* g, int n, const int* type) {
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_set_source_types: grid is NULL");
  if (n != (int)g->src.size())
    return fail(RT_ERR_INVALID_ARG, "rt_set_source_types: n = %d, the grid has %zu sources", n, g->src.size());
  if (n > 0 && !type) return fail(RT_ERR_INVALID_ARG, "rt_set_source_types: type is NULL");
  for (int i = 0; i < n; ++i) {
    if (type[i] < 0 || type[i] >= kTypes) return fail(RT_ERR_INVALID_ARG, "rt_set_source_types: type[%d] = %d", i, type[i]);
    if (!(g->src[i].e_ph >= kEIon[type[i]]))
      return fail(RT_ERR_INVALID_ARG, "rt_set_source_types: source %d: %g eV is below the %g eV threshold", i,
                  g->src[i].e_ph, kEIon[type[i]]);
  }
  for (int i = 0; i < n; ++i) g->src[i].type = type[i];
  g->src_dirty = true;
  mark_batch_dirty(g);
  return RT_OK;
}

int rt_get_rates(rt_grid* g, void* kph, void* gamma, void* x_HI, int dtype, int mem_kind) {
  NvtxRange nr("rt_get_rates");
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_get_rates: grid is NULL");
  if (int rcw = wait_batch(g)) return rcw;
  if (dtype != RT_DTYPE_F64 && dtype != RT_DTYPE_F32) return fail(RT_ERR_INVALID_ARG, "rt_get_rates: dtype %d", dtype);
  if (mem_kind != RT_MEM_HOST && mem_kind != RT_MEM_DEVICE) return fail(RT_ERR_INVALID_ARG, "rt_get_rates: mem_kind %d", mem_kind);
  CUDA_TRY(cudaSetDevice(g->ctx->device));
  const int kd = g->precision == RT_FP64 ? RT_DTYPE_F64 : RT_DTYPE_F32;
  int rc;
  if ((rc = copy_field(g, g->K, kd, kph, dtype, mem_kind))) return rc;
  if ((rc = copy_field(g, g->G, kd, gamma, dtype, mem_kind, gamma_scale(g)))) return rc;
  if ((rc = copy_field(g, g->xHI, RT_DTYPE_F64, x_HI, dtype, mem_kind))) return rc;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return RT_OK;
}

int rt_get_rates_typed(rt_grid* g, int type, void* kph, void* gamma, int dtype, int mem_kind) {
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_get_rates_typed: grid is NULL");
  if (type < 0 || type >= kTypes) return fail(RT_ERR_INVALID_ARG, "rt_get_rates_typed: type %d", type);
  if (type == 0) return rt_get_rates(g, kph, gamma, nullptr, dtype, mem_kind);
  if (int rcw = wait_batch(g)) return rcw;
  if (!g->he) return fail(RT_ERR_INVALID_ARG, "rt_get_rates_typed: the grid has no helium absorbers");
  if (dtype != RT_DTYPE_F64 && dtype != RT_DTYPE_F32) return fail(RT_ERR_INVALID_ARG, "rt_get_rates_typed: dtype %d", dtype);
  if (mem_kind != RT_MEM_HOST && mem_kind != RT_MEM_DEVICE)
    return fail(RT_ERR_INVALID_ARG, "rt_get_rates_typed: mem_kind %d", mem_kind);
  CUDA_TRY(cudaSetDevice(g->ctx->device));
  const int kd = g->precision == RT_FP64 ? RT_DTYPE_F64 : RT_DTYPE_F32;
  int rc;
  if ((rc = copy_field(g, g->Khe[type - 1], kd, kph, dtype, mem_kind))) return rc;
  if ((rc = copy_field(g, g->Ghe[type - 1], kd, gamma, dtype, mem_kind, gamma_scale(g)))) return rc;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return RT_OK;
}

int rt_set_rates(rt_grid* g, const void* kph, const void* gamma, int dtype, int mem_kind) {
  if (!g || !kph || !gamma) return fail(RT_ERR_INVALID_ARG, "rt_set_rates: grid, kph and gamma are required");
  if (int rcw = wait_batch(g)) return rcw;
  if (dtype != RT_DTYPE_F64 && dtype != RT_DTYPE_F32) return fail(RT_ERR_INVALID_ARG, "rt_set_rates: dtype %d", dtype);
  if (mem_kind != RT_MEM_HOST && mem_kind != RT_MEM_DEVICE) return fail(RT_ERR_INVALID_ARG, "rt_set_rates: mem_kind %d", mem_kind);
  CUDA_TRY(cudaSetDevice(g->ctx->device));
  const long long n = g->ncell;
  const size_t eb = dtype == RT_DTYPE_F64 ? 8 : 4;
  const int kd = g->precision == RT_FP64 ? RT_DTYPE_F64 : RT_DTYPE_F32;
  cudaStream_t st = g->stream;
  const void* src[2] = {kph, gamma};
  void* dst[2] = {g->K, g->G};
  const double scale[2] = {1.0, 1.0 / gamma_scale(g)};
  for (int f = 0; f < 2; ++f) {
    if (mem_kind == RT_MEM_DEVICE) {
      LAUNCH_TRY(launch_convert(n, src[f], dtype, dst[f], kd, st, scale[f]));
      continue;
    }
    void* tmp = nullptr;
    CUDA_TRY(cudaMallocAsync(&tmp, (size_t)n * eb, st));
    cudaError_t e = cudaMemcpyAsync(tmp, src[f], (size_t)n * eb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_convert(n, tmp, dtype, dst[f], kd, st, scale[f]);
    if (e == cudaSuccess) g_launches.fetch_add(1);
    cudaFreeAsync(tmp, st);
    if (e != cudaSuccess) return fail(RT_ERR_CUDA, "rt_set_rates: %s", cudaGetErrorString(e));
  }
  if (mem_kind == RT_MEM_HOST) CUDA_TRY(cudaStreamSynchronize(st));
  return RT_OK;
}

int rt_timestep(rt_grid* g, double eps_ion, double alpha_B, double sigma_front, double tau_front, double dt_max,
                double dt_prev, double* dt_out) {
  if (!g || !dt_out) return fail(RT_ERR_INVALID_ARG, "rt_timestep: grid and dt_out are required");
  if (!(eps_ion > 0) || !isfinite(eps_ion) || !(alpha_B >= 0) || !isfinite(alpha_B) || !(sigma_front >= 0) ||
      !isfinite(sigma_front) || !(tau_front >= 0) || !(dt_max > 0) || !(dt_prev >= 0))
    return fail(RT_ERR_INVALID_ARG, "rt_timestep: bad parameter");
  if (int rcw = wait_batch(g)) return rcw;
  CUDA_TRY(cudaSetDevice(g->ctx->device));
  cudaStream_t st = g->stream;
  const long long n = g->ncell;
  char* scratch = nullptr;
  CUDA_TRY(cudaMallocAsync((void**)&scratch, (size_t)n * sizeof(float) + 256, st));
  unsigned int* out = (unsigned int*)(scratch + (((size_t)n * sizeof(float) + 255) & ~(size_t)255));
  unsigned int* h = (unsigned int*)((char*)g->host_rb + 3072);
  *h = 0x7f800000u;  // +inf
  cudaError_t e = cudaMemcpyAsync(out, h, sizeof *h, cudaMemcpyHostToDevice, st);
  // finite dt_max: values in units of dt_max (cells outside the front hold 1)
  const bool finite = isfinite(dt_max) && dt_max < 3.0e38;
  const float dmax = finite ? (float)dt_max : 3.0e38f;
  if (e == cudaSuccess)
    e = launch_timestep(n, g->nx, g->ny, g->nz, g->nH, g->xHI, g->K, g->precision == RT_FP64,
                        sigma_front * g->dx, tau_front, (float)eps_ion, (float)alpha_B, dmax, finite ? dmax : 1.0f,
                        (float*)scratch, out, st);
  if (e == cudaSuccess) g_launches.fetch_add(2);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, sizeof *h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, "rt_timestep: %s", cudaGetErrorString(e));
  float v;
  memcpy(&v, h, sizeof v);
  double dt = finite ? (v >= 1.0f ? dt_max : (double)v * dt_max) : (v >= 3.0e38f ? dt_max : (double)v);
  if (dt_prev > 0 && 2.0 * dt_prev < dt) dt = 2.0 * dt_prev;  // Eq. "dtchange"
  *dt_out = dt;
  return RT_OK;
}

int rt_get_in_flight(rt_grid* g, rt_flight* out, uint64_t cap, uint64_t* n) {
  if (!g || !n || (cap > 0 && !out)) return fail(RT_ERR_INVALID_ARG, "rt_get_in_flight: NULL argument");
  if (int rcw = wait_batch(g)) return rcw;
  CUDA_TRY(cudaSetDevice(g->ctx->device));
  *n = 0;
  if (!g->fl.live) return RT_OK;
  unsigned long long cnt = 0;
  CUDA_TRY(cudaMemcpyAsync(&cnt, g->ts.ctl + CTL_HALTED, sizeof cnt, cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  const FlightState& F = g->fl;
  const unsigned long long stored = cnt < F.cap[F.in] ? cnt : F.cap[F.in];
  *n = stored;
  const unsigned long long m = stored < cap ? stored : cap;
  if (m == 0) return RT_OK;
  const bool f64 = g->precision == RT_FP64;
  const size_t rec = f64 ? sizeof(Rec64) : sizeof(Rec32);
  std::vector<unsigned char> raw((size_t)m * rec);
  CUDA_TRY(cudaMemcpyAsync(raw.data(), F.buf[F.in], raw.size(), cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  const unsigned nx = (unsigned)g->nx, ny = (unsigned)g->ny;
  for (unsigned long long i = 0; i < m; ++i) {
    rt_flight& o = out[i];
    memset(&o, 0, sizeof o);
    uint32_t cell;
    double P;
    if (f64) {
      const Rec64& q = ((const Rec64*)raw.data())[i];
      o.r_cm = q.r * g->dx;
      P = q.P;
      o.tau = q.tau;
      o.src = (int32_t)q.src;
      o.level = (int32_t)(q.level & 15u);
      o.pix = q.pix;
      o.age = q.level >> 4;
      cell = q.tag;
    } else {
      const Rec32& q = ((const Rec32*)raw.data())[i];
      o.r_cm = ((double)q.r + (double)q.r_lo) * g->dx;
      P = q.P;
      o.tau = (double)q.tau + (double)q.tau_lo;
      o.src = (int32_t)q.src;
      o.level = (int32_t)(q.tag & 15u);
      o.pix = q.pix;
      o.age = q.age;
      cell = q.cell;
    }
    o.P = (size_t)o.src < F.unit.size() ? P * F.unit[o.src] : 0.0;
    o.cell[0] = (int32_t)(cell % nx);
    o.cell[1] = (int32_t)((cell / nx) % ny);
    o.cell[2] = (int32_t)(cell / (nx * ny));
  }
  return RT_OK;
}

int rt_get_ionised(rt_grid* g, void* x_HII, int dtype, int mem_kind) {
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_get_ionised: grid is NULL");
  if (int rcw = wait_batch(g)) return rcw;
  if (dtype != RT_DTYPE_F64 && dtype != RT_DTYPE_F32) return fail(RT_ERR_INVALID_ARG, "rt_get_ionised: dtype %d", dtype);
  if (mem_kind != RT_MEM_HOST && mem_kind != RT_MEM_DEVICE) return fail(RT_ERR_INVALID_ARG, "rt_get_ionised: mem_kind %d", mem_kind);
  CUDA_TRY(cudaSetDevice(g->ctx->device));
  int rc = copy_field(g, g->xHII, RT_DTYPE_F64, x_HII, dtype, mem_kind);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return RT_OK;
}

int rt_selfcheck_directions(rt_ctx* ctx, int level, double* max_abs_err, double* bound) {
  if (!ctx || !max_abs_err || level < 0 || level > RT_MAX_LEVEL)
    return fail(RT_ERR_INVALID_ARG, "rt_selfcheck_directions: bad argument");
  CUDA_TRY(cudaSetDevice(ctx->device));
  unsigned long long* d = nullptr;
  CUDA_TRY(cudaMalloc(&d, sizeof *d));
  cudaError_t e = cudaMemset(d, 0, sizeof *d);
  if (e == cudaSuccess) e = launch_direction_check(level, d, 0);
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, "rt_selfcheck_directions: %s", cudaGetErrorString(e));
  g_launches.fetch_add(1);
  double v;
  memcpy(&v, &h, sizeof v);
  *max_abs_err = v;
  if (bound) *bound = (double)kDirErr32;
  return RT_OK;
}

int rt_synchronize(rt_grid* g) {
  if (!g) return fail(RT_ERR_INVALID_ARG, "rt_synchronize: grid is NULL");
  if (int rcw = wait_batch(g)) return rcw;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (g->up) CUDA_TRY(cudaStreamSynchronize(g->up));
  if (g->dn) CUDA_TRY(cudaStreamSynchronize(g->dn));
  if (g->ev_commit) {
    // a state uploaded by rt_set_state_async may have been rejected
    unsigned long long* h = (unsigned long long*)((char*)g->host_rb + 3584);
    CUDA_TRY(cudaMemcpyAsync(h, g->ts.ctl + CTL_SET_ERR, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (h[0]) {
      note_rejected_state(g, h[1], h[2]);
      CUDA_TRY(cudaStreamSynchronize(g->stream));
      return fail(RT_ERR_INVALID_ARG, "rt_synchronize: %s", g->set_err.c_str());
    }
  }
  return RT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many grids traced by one persistent launch (one global queue; each
// grid keeps its own fields, budget and counters).
// ---------------------------------------------------------------------------
struct rt_batch {
  rt_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int precision = -1;
  std::vector<rt_grid*> slots;  // nullptr = free slot
  // device tables of the active grids (compact, in slot order)
  std::vector<int> dev_slot;    // device instance index -> slot
  InstDev* inst_dev = nullptr;
  size_t inst_cap = 0;
  SourceDev* src_dev = nullptr;
  size_t src_cap = 0;
  int nsrc = 0;
  unsigned long long n_roots = 0;
  long long max_cells = 0;
  int max_dims = 0;
  double max_diag = 0;
  bool dirty = true;
  int built_level0 = -1;
  TraceState ts;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool traced = false;
  void* host_rb = nullptr;
  // captured step graph and the arguments it was captured with
  cudaGraphExec_t graph = nullptr;
  bool graph_ok = false;
  unsigned long long graph_launches = 0;  // kernels one replay runs
  rt_trace_params gp;
  double g_dt = 0, g_alpha = 0;
  int g_nsub = 0;
  ~rt_batch() {
    if (graph) cudaGraphExecDestroy(graph);
    if (inst_dev) cudaFree(inst_dev);
    if (src_dev) cudaFree(src_dev);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (host_rb) cudaFreeHost(host_rb);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};


static int batch_rebuild(rt_batch* b, int level0) {
  if (!b->dirty && b->built_level0 == level0) return RT_OK;
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  std::vector<InstDev> inst;
  std::vector<SourceDev> src;
  b->dev_slot.clear();
  b->max_cells = 0;
  b->max_dims = 0;
  double diag = 0;
  for (size_t s = 0; s < b->slots.size(); ++s) {
    rt_grid* g = b->slots[s];
    if (!g) continue;
    for (const rt_grid::SrcIn& S : g->src)
      if (S.type > 0 && !g->he)
        return fail(RT_ERR_INVALID_ARG, "batch: slot %zu has helium photon types but no rt_set_absorbers", s);
    const InstDev I = inst_of(g);
    build_sources(g, level0, (int)inst.size(), src);
    inst.push_back(I);
    b->dev_slot.push_back((int)s);
    if (g->ncell > b->max_cells) b->max_cells = g->ncell;
    const int ds = g->nx + g->ny + g->nz;
    if (ds > b->max_dims) b->max_dims = ds;
    const double d = sqrt((double)g->nx * g->nx + (double)g->ny * g->ny + (double)g->nz * g->nz);
    if (d > diag) diag = d;
  }
  if (inst.size() > b->inst_cap) {
    if (b->inst_dev) cudaFree(b->inst_dev);
    b->inst_dev = nullptr;
    b->inst_cap = 0;
    CUDA_TRY(cudaMalloc((void**)&b->inst_dev, inst.size() * sizeof(InstDev)));
    b->inst_cap = inst.size();
  }
  if (src.size() > b->src_cap) {
    if (b->src_dev) cudaFree(b->src_dev);
    b->src_dev = nullptr;
    b->src_cap = 0;
    CUDA_TRY(cudaMalloc((void**)&b->src_dev, src.size() * sizeof(SourceDev)));
    b->src_cap = src.size();
  }
  // on the batch's stream (which may not be ordered with the legacy stream);
  // the host vectors live until the copies end
  if (!inst.empty())
    CUDA_TRY(cudaMemcpyAsync(b->inst_dev, inst.data(), inst.size() * sizeof(InstDev), cudaMemcpyHostToDevice, b->stream));
  if (!src.empty())
    CUDA_TRY(cudaMemcpyAsync(b->src_dev, src.data(), src.size() * sizeof(SourceDev), cudaMemcpyHostToDevice, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  b->nsrc = (int)src.size();
  b->n_roots = (12ULL << (2 * level0)) * (unsigned long long)src.size();
  b->max_diag = diag;
  b->dirty = false;
  b->built_level0 = level0;
  b->graph_ok = false;
  return RT_OK;
}

static int batch_enqueue(rt_batch* b, const rt_trace_params* p, int passes) {
  int rc = batch_rebuild(b, p->level0);
  if (rc) return rc;
  const int ninst = (int)b->dev_slot.size();
  cudaStream_t st = b->stream;
  LAUNCH_TRY(launch_batch_zero(b->inst_dev, ninst, b->precision, b->max_cells, st));  // Step 2
  if (b->nsrc == 0) {
    LAUNCH_TRY(launch_trace_init(b->ts.ctl, b->ts.queue, b->ts.cap * b->ts.rec_bytes, 0, 1, FLIGHT_OFF, 0, 0, 1, st));
    b->traced = false;
    b->ts.passes_run = 0;
    return RT_OK;
  }
  TraceArgs A;
  memset(&A, 0, sizeof A);
  fill_common_args(A, p);
  A.inst = b->inst_dev;
  A.ninst = ninst;
  A.npix0 = (uint32_t)(12u << (2 * p->level0));
  A.queue = b->ts.queue;
  A.cap = b->ts.cap;
  A.ctl = b->ts.ctl;
  A.max_steps = 2 * b->max_dims + 16;
  A.dir_tab = nullptr;
  A.dir_levels = -1;
  if (b->precision == RT_FP32_MIXED) {
    // deepest level a package can reach in the largest grid
    int want = p->level0;
    while (want < p->max_level && A.rsplit[want] < b->max_diag) ++want;
    if (want > kDirTableMaxLevel) want = kDirTableMaxLevel;
    if ((rc = ensure_dir_table(b->ctx, want, &A.dir_tab, &A.dir_levels))) return rc;
  }
  int per_sm = 0;
  CUDA_TRY(trace_occupancy(b->precision, 0, 256, &per_sm));
  if (per_sm < 1) per_sm = 1;
  if (p->blocks_per_sm > 0 && p->blocks_per_sm < per_sm) per_sm = p->blocks_per_sm;
  if ((rc = b->ts.bind_rows(A, per_sm * b->ctx->num_sms, ninst))) return rc;
  if ((rc = launch_passes(A, b->ts.cap * b->ts.rec_bytes, b->src_dev, b->nsrc, passes, b->precision, 0, FLIGHT_OFF, 0,
                          per_sm * b->ctx->num_sms,
                          b->ev0, b->ev1, st)))
    return rc;
  b->traced = true;
  b->ts.passes_run = passes < b->nsrc ? passes : b->nsrc;
  return RT_OK;
}

static int batch_ensure_queue(rt_batch* b, unsigned long long cap) {
  const size_t rec = queue_rec_bytes(b->precision == RT_FP64, false);
  if (b->ts.queue && b->ts.cap >= cap && b->ts.rec_bytes == rec) return RT_OK;
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  if (b->ts.queue) cudaFree(b->ts.queue);
  b->ts.queue = nullptr;
  b->ts.cap = 0;
  CUDA_TRY(cudaMalloc(&b->ts.queue, cap * rec));
  CUDA_TRY(cudaMemsetAsync(b->ts.queue, 0, cap * rec, b->stream));
  b->ts.cap = cap;
  b->ts.rec_bytes = rec;
  b->graph_ok = false;
  return RT_OK;
}

// status and queue use of the batch's last trace (synchronises)
struct BatchStatus {
  int status;
  unsigned long long pushed;  // records, all passes
  unsigned long long peak;    // records of the largest pass
  float ms;
};

static int batch_status(rt_batch* b, BatchStatus* bs) {
  unsigned long long* hctl = (unsigned long long*)b->host_rb;
  CUDA_TRY(cudaMemcpyAsync(hctl, b->ts.ctl, CTL_N * sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  bs->status = (int)hctl[CTL_STATUS];
  bs->pushed = hctl[CTL_PUSHED] + hctl[CTL_TAIL];
  bs->peak = hctl[CTL_PEAK] > hctl[CTL_TAIL] ? hctl[CTL_PEAK] : hctl[CTL_TAIL];
  bs->ms = 0.f;
  if (b->traced && cudaEventElapsedTime(&bs->ms, b->ev0, b->ev1) != cudaSuccess) {
    bs->ms = 0.f;
    cudaGetLastError();
  }
  return RT_OK;
}

// A member's sources or absorbers changed: the batch's source and grid
// tables (and a captured step) no longer describe it.
static void mark_batch_dirty(rt_grid* g) {
  if (g->batch) g->batch->dirty = true;
}

static void detach_grid(rt_grid* g) {
  rt_batch* b = g->batch;
  b->slots[g->batch_slot] = nullptr;
  b->dirty = true;
  bool any = false;
  for (rt_grid* h : b->slots) any |= h != nullptr;
  if (!any) b->precision = -1;
  g->batch = nullptr;
  g->batch_slot = -1;
  g->batch_stream = nullptr;
}

extern "C" {

int rt_batch_create(rt_ctx* ctx, void* stream, rt_batch** out) {
  if (!ctx || !out) return fail(RT_ERR_INVALID_ARG, "rt_batch_create: NULL argument");
  CUDA_TRY(cudaSetDevice(ctx->device));
  rt_batch* b = new rt_batch;
  b->ctx = ctx;
  cudaError_t e = cudaSuccess;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreate(&b->stream);  // blocking: ordered with the legacy default stream
    b->own_stream = true;
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->ts.ctl, CTL_N * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ts.ctl, 0, CTL_N * sizeof(unsigned long long), b->stream);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->ts.blk, blk_rows_bytes(ctx->num_sms, kBlkGrids));
  if (e == cudaSuccess) {
    b->ts.blk_blocks = ctx->num_sms * kBlkMaxPerSM;
    b->ts.blk_rows = kBlkGrids;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
  if (e == cudaSuccess) e = cudaMallocHost(&b->host_rb, 4096);
  if (e != cudaSuccess) {
    delete b;
    return fail(RT_ERR_CUDA, "rt_batch_create: %s", cudaGetErrorString(e));
  }
  *out = b;
  return RT_OK;
}

int rt_batch_destroy(rt_batch* b) {
  if (!b) return RT_OK;
  cudaStreamSynchronize(b->stream);
  for (rt_grid* g : b->slots)
    if (g) {
      g->batch = nullptr;
      g->batch_slot = -1;
      g->batch_stream = nullptr;
    }
  delete b;
  return RT_OK;
}

int rt_batch_add(rt_batch* b, rt_grid* g, int* slot) {
  if (!b || !g || !slot) return fail(RT_ERR_INVALID_ARG, "rt_batch_add: NULL argument");
  if (g->ctx != b->ctx) return fail(RT_ERR_INVALID_ARG, "rt_batch_add: grid belongs to another context");
  if (b->precision >= 0 && g->precision != b->precision)
    return fail(RT_ERR_INVALID_ARG, "rt_batch_add: every grid of a batch has the same precision");
  if (g->batch) return fail(RT_ERR_STATE, "rt_batch_add: grid is already in a batch");
  CUDA_TRY(cudaStreamSynchronize(g->stream));  // work already queued on the grid's own stream
  drop_flight(g);  // batches trace with an infinite speed of light
  b->precision = g->precision;
  int s = -1;
  for (size_t i = 0; i < b->slots.size(); ++i)
    if (!b->slots[i]) { s = (int)i; break; }
  if (s < 0) {
    s = (int)b->slots.size();
    b->slots.push_back(nullptr);
  }
  b->slots[s] = g;
  g->batch = b;
  g->batch_slot = s;
  g->batch_stream = b->stream;
  b->dirty = true;
  *slot = s;
  return RT_OK;
}

int rt_batch_remove(rt_batch* b, int slot) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot])
    return fail(RT_ERR_INVALID_ARG, "rt_batch_remove: no grid in slot %d", slot);
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  detach_grid(b->slots[slot]);
  return RT_OK;
}

int rt_batch_size(rt_batch* b) {
  if (!b) return 0;
  int n = 0;
  for (rt_grid* h : b->slots) n += h != nullptr;
  return n;
}

// per-grid calls (rt_set_state, rt_trace, ...) run on each grid's own stream;
// a batch launch reads every member, so it starts after them
static int sync_members(rt_batch* b) {
  for (rt_grid* g : b->slots)
    if (g) CUDA_TRY(cudaStreamSynchronize(g->stream));
  return RT_OK;
}

// Batches trace with an infinite speed of light only.
static int check_batch_params(const rt_trace_params* p) {
  int rc = check_params(p);
  if (rc) return rc;
  if (p->light_cm != 0.0) return fail(RT_ERR_INVALID_ARG, "batch traces take light_cm = 0 (infinite speed of light)");
  return RT_OK;
}

int rt_batch_trace(rt_batch* b, const rt_trace_params* p, int sync) {
  NvtxRange nr("rt_batch_trace");
  if (!b) return fail(RT_ERR_INVALID_ARG, "rt_batch_trace: batch is NULL");
  int rc = check_batch_params(p);
  if (rc) return rc;
  CUDA_TRY(cudaSetDevice(b->ctx->device));
  if (rt_batch_size(b) == 0) return RT_OK;
  if ((rc = sync_members(b))) return rc;
  unsigned long long cap = (unsigned long long)p->queue_capacity;
  const bool automatic = cap == 0;
  if (automatic) {
    cap = b->ts.cap;
    if (cap == 0) {
      long long cells = 0;
      for (rt_grid* g : b->slots) if (g) cells += g->ncell;
      cap = (unsigned long long)cells * 2ULL;
      if (cap < (1ULL << 20)) cap = 1ULL << 20;
      if (cap > (1ULL << 26)) cap = 1ULL << 26;
    }
  }
  const size_t rec = queue_rec_bytes(b->precision == RT_FP64, false);
  const int p_min = p->passes > 1 ? p->passes : 1;
  int passes = automatic && b->ts.passes > p_min ? b->ts.passes : p_min;
  for (int attempt = 0;; ++attempt) {
    if ((rc = batch_ensure_queue(b, cap))) return rc;
    if ((rc = batch_enqueue(b, p, passes))) return rc;
    if (!sync) return RT_OK;
    BatchStatus bs;
    if ((rc = batch_status(b, &bs))) return rc;
    if (bs.status == RT_ERR_QUEUE_OVERFLOW && automatic && attempt < 40) {
      const unsigned long long limit = queue_cap_limit(rec, (size_t)b->ts.cap * b->ts.rec_bytes);
      if (grow_after_overflow(bs.peak, limit, b->nsrc, &cap, &passes)) continue;
    }
    if (bs.status != RT_OK)
      return fail(bs.status, "rt_batch_trace: device status %d (queue capacity %llu, largest pass %llu, passes %d)",
                  bs.status, (unsigned long long)b->ts.cap, bs.peak, b->ts.passes_run);
    if (automatic && passes > p_min) b->ts.passes = 4 * bs.peak < b->ts.cap ? passes / 2 : passes;
    return RT_OK;
  }
}

int rt_batch_chem(rt_batch* b, double dt_s, int nsub, double alpha_B) {
  if (!b) return fail(RT_ERR_INVALID_ARG, "rt_batch_chem: batch is NULL");
  if (!(dt_s >= 0) || !isfinite(dt_s) || nsub < 1 || !(alpha_B >= 0) || !isfinite(alpha_B))
    return fail(RT_ERR_INVALID_ARG, "rt_batch_chem: bad dt_s / nsub / alpha_B");
  CUDA_TRY(cudaSetDevice(b->ctx->device));
  if (rt_batch_size(b) == 0) return RT_OK;
  if (int rcs = sync_members(b)) return rcs;
  if (b->dirty) {
    int rc = batch_rebuild(b, b->built_level0 >= 0 ? b->built_level0 : 1);
    if (rc) return rc;
  }
  LAUNCH_TRY(launch_batch_chem(b->inst_dev, (int)b->dev_slot.size(), b->precision, b->max_cells, dt_s / nsub, nsub,
                               alpha_B, b->stream));
  return RT_OK;
}

static bool same_params(const rt_trace_params& a, const rt_trace_params& b) {
  return a.level0 == b.level0 && a.phi_c == b.phi_c && a.f_term == b.f_term && a.max_level == b.max_level &&
         a.queue_capacity == b.queue_capacity && a.timeout_s == b.timeout_s && a.blocks_per_sm == b.blocks_per_sm &&
         a.segs_per_iter == b.segs_per_iter && a.flags == b.flags && a.passes == b.passes;
}

int rt_batch_step(rt_batch* b, const rt_trace_params* p, double dt_s, int nsub, double alpha_B, int nsteps) {
  NvtxRange nr("rt_batch_step");
  if (!b) return fail(RT_ERR_INVALID_ARG, "rt_batch_step: batch is NULL");
  int rc = check_batch_params(p);
  if (rc) return rc;
  if (nsteps < 0 || !(dt_s >= 0) || !isfinite(dt_s) || nsub < 1 || !(alpha_B >= 0) || !isfinite(alpha_B))
    return fail(RT_ERR_INVALID_ARG, "rt_batch_step: bad nsteps / dt_s / nsub / alpha_B");
  CUDA_TRY(cudaSetDevice(b->ctx->device));
  if (rt_batch_size(b) == 0 || nsteps == 0) return RT_OK;
  if ((rc = sync_members(b))) return rc;
  const bool reuse = b->graph_ok && !b->dirty && b->built_level0 == p->level0 && same_params(b->gp, *p) &&
                     b->g_dt == dt_s && b->g_nsub == nsub && b->g_alpha == alpha_B;
  if (!reuse) {
    // size the queue (and build tables) with one synchronous trace, then
    // capture one step -- zero, emit, trace, update -- as a graph
    rt_trace_params q = *p;
    if ((rc = rt_batch_trace(b, &q, 1))) return rc;
    const int passes = b->ts.passes_run > 0 ? b->ts.passes_run : 1;
    if (q.queue_capacity == 0) {
      BatchStatus bs;
      if ((rc = batch_status(b, &bs))) return rc;
      // headroom: the media evolve between replays, and traces grow as they ionise
      const size_t rec = queue_rec_bytes(b->precision == RT_FP64, false);
      const unsigned long long limit = queue_cap_limit(rec, (size_t)b->ts.cap * b->ts.rec_bytes);
      unsigned long long need = 4 * bs.peak + (1ULL << 20);
      if (need > limit) need = limit;
      if (need > b->ts.cap && (rc = batch_ensure_queue(b, need))) return rc;
      q.queue_capacity = (int64_t)b->ts.cap;
    }
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaGraph_t graph = nullptr;
    const unsigned long long launches_before = g_launches.load();
    CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc1 = batch_enqueue(b, &q, passes);
    cudaError_t e1 = launch_batch_chem(b->inst_dev, (int)b->dev_slot.size(), b->precision, b->max_cells,
                                       dt_s / nsub, nsub, alpha_B, b->stream);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    b->graph_launches = g_launches.load() - launches_before + 1;  // + the update
    g_launches.store(launches_before);  // captured kernels count when the graph runs
    if (rc1) { if (graph) cudaGraphDestroy(graph); return rc1; }
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail(RT_ERR_CUDA, "rt_batch_step: capture: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    }
    cudaError_t e3 = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) return fail(RT_ERR_CUDA, "rt_batch_step: instantiate: %s", cudaGetErrorString(e3));
    b->graph_ok = true;
    b->gp = *p;
    b->g_dt = dt_s;
    b->g_nsub = nsub;
    b->g_alpha = alpha_B;
  }
  for (int i = 0; i < nsteps; ++i) {
    CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
    g_launches.fetch_add(b->graph_launches);
  }
  return RT_OK;
}

int rt_batch_get_budget(rt_batch* b, int slot, rt_budget* out) {
  if (!b || !out || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot])
    return fail(RT_ERR_INVALID_ARG, "rt_batch_get_budget: no grid in slot %d", slot);
  BatchStatus bs;
  int rc = batch_status(b, &bs);
  if (rc) return rc;
  const int status = bs.status;
  rt_grid* g = b->slots[slot];
  double* hacc = (double*)g->host_rb;
  unsigned long long* hcnt = (unsigned long long*)((char*)g->host_rb + 64);
  CUDA_TRY(cudaMemcpyAsync(hacc, g->acc, kAccWords * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaMemcpyAsync(hcnt, g->cnt, kCntWords * sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  memset(out, 0, sizeof *out);
  out->emitted = hacc[0];
  out->absorbed = hacc[1];
  out->escaped = hacc[2];
  for (int l = 0; l < kLevels; ++l) {
    out->counts[l] = hcnt[l];
    out->hashes[l] = hcnt[kLevels + l];
  }
  out->segments = hcnt[kCntSegments];
  out->fallbacks = hcnt[kCntFallbacks];
  out->fallbacks_tau = hcnt[kCntFallbacksTau];
  out->queue_pushed = bs.pushed;
  out->queue_peak = bs.peak;
  out->passes = b->ts.passes_run;
  out->status = status;
  out->kernel_ms = bs.ms;
  if (status != RT_OK) return fail(status, "rt_batch_get_budget: device status %d", status);
  return RT_OK;
}

int rt_batch_autotune(rt_batch* b, rt_trace_params* p) {
  if (!b || !p) return fail(RT_ERR_INVALID_ARG, "rt_batch_autotune: NULL argument");
  int rc = check_batch_params(p);
  if (rc) return rc;
  if (rt_batch_size(b) == 0) return RT_OK;
  rt_trace_params q = *p;
  q.segs_per_iter = 8;
  q.blocks_per_sm = 0;
  if ((rc = rt_batch_trace(b, &q, 1))) return rc;  // sizes the queue, warms up
  const int spi[] = {4, 8, 16, 32, 64};
  int per_sm_max = 0;
  CUDA_TRY(trace_occupancy(b->precision, 0, 256, &per_sm_max));
  float best = 1e30f;
  rt_trace_params bestp = q;
  for (int bps = 1; bps <= (per_sm_max > 0 ? per_sm_max : 1); ++bps) {
    for (int s : spi) {
      q.segs_per_iter = s;
      q.blocks_per_sm = bps;
      float tmin = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        if ((rc = rt_batch_trace(b, &q, 1))) return rc;
        BatchStatus bs;
        if ((rc = batch_status(b, &bs))) return rc;
        if (bs.ms < tmin) tmin = bs.ms;
      }
      if (tmin < best) {
        best = tmin;
        bestp = q;
      }
    }
  }
  p->segs_per_iter = bestp.segs_per_iter;
  p->blocks_per_sm = bestp.blocks_per_sm;
  return RT_OK;
}

}  // extern "C"
