// noalloc.cu -- rt_trace_noalloc: the FP32-mixed trace with no device memory
// allocation at all.
//
// Some callers cannot allocate device memory: applications whose device
// memory is owned by a host framework (an arena or a caching allocator with a
// fixed budget) and callers that must not let cudaMalloc/cudaFree synchronise
// the device or change its memory footprint.  For them this entry point keeps
// all of the trace's scratch -- package queue, control words, photon-budget
// sums, source records and the table of pixel directions -- in one file-scope
// static device array of fixed size; the caller passes device pointers for the
// inputs and outputs.
//
// The array exists once per device that loads the library and stays until the
// process exits.  Every call shares it: calls whose work overlaps on the GPU
// (different streams, or several host threads) race on it and must be
// serialised by the caller.  Each call clears the parts that must start at
// zero; the rest keeps the last call's contents.  The first call on a device
// does the per-device set-up (looks up the array's device address and fills
// the direction table) and synchronises that device; make that first call
// before any stream capture.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>

#include "rt.h"
#include "rt_internal.cuh"

namespace rtg {
cudaError_t launch_trace_init(unsigned long long* ctl, void* queue, size_t queue_bytes, unsigned long long n_roots,
                              int first_pass, int mode, unsigned long long in_cap, int pass, int passes,
                              cudaStream_t st);
cudaError_t trace_occupancy(int precision, int fsl, int block, int* blocks_per_sm);
cudaError_t launch_trace(int precision, int fsl, const TraceArgs& A, int grid, int block, cudaStream_t st);
cudaError_t launch_direction_table(int level, float4* tab, cudaStream_t st);
}  // namespace rtg

using namespace rtg;

namespace {

// Layout of the static scratch (byte offsets, each 256-byte aligned).
constexpr size_t na_align(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr int kNaTableLevels = 6;  // directions of levels 0..6 (deeper levels: FP64 on the fly)
constexpr size_t kNaTableEntries = 4 * ((size_t(1) << (2 * (kNaTableLevels + 1))) - 1);
constexpr size_t kNaCtlOff = 0;     // CTL_N control words
constexpr size_t kNaAccOff = 512;   // kNaAccWords doubles (the trace's budget sums)
constexpr size_t kNaCntOff = 640;   // kCntWords counters
constexpr int kNaAccWords = 8;      // emitted, absorbed, escaped, resumed, halted; spare
constexpr size_t kNaInstOff = 1024; // one InstDev
constexpr size_t kNaSrcOff = 2048;  // RT_NOALLOC_MAX_SOURCES SourceDev
constexpr size_t kNaTabOff = na_align(kNaSrcOff + (size_t)RT_NOALLOC_MAX_SOURCES * sizeof(SourceDev));
constexpr size_t kNaQueueOff = na_align(kNaTabOff + kNaTableEntries * 2 * sizeof(float4));
constexpr size_t kNaQueueBytes = (size_t)RT_NOALLOC_MAX_RECORDS * sizeof(QRec32);
constexpr int kNaMaxBlocks = 2048;  // trace blocks the budget rows are laid out for
constexpr size_t kNaBlkOff = na_align(kNaQueueOff + kNaQueueBytes);
constexpr size_t kNaBytes = kNaBlkOff + (size_t)kNaMaxBlocks * kBlkRow * sizeof(double);
static_assert(CTL_N * 8 <= kNaAccOff && kNaAccOff + kNaAccWords * 8 <= kNaCntOff && kNaCntOff + kCntWords * 8 <= kNaInstOff &&
                  sizeof(InstDev) <= kNaSrcOff - kNaInstOff,
              "scratch layout");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
unsigned char* g_na_ptr[kNaMaxDevices];  // device address of the scratch, per device
int g_na_sms[kNaMaxDevices];

thread_local std::string g_na_error;

int na_fail(int code, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[512];
  snprintf(buf, sizeof buf, "rt_trace_noalloc: %s%s%s", msg, e != cudaSuccess ? ": " : "",
           e != cudaSuccess ? cudaGetErrorString(e) : "");
  g_na_error = buf;
  return code;
}

// Per-device set-up, with the device current: the scratch's device address
// and the direction table.  Synchronises the device the first time.
int na_setup(int dev, unsigned char** base, int* sms) {
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (dev < 0 || dev >= kNaMaxDevices) return na_fail(RT_ERR_INVALID_ARG, "device index out of range");
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return na_fail(RT_ERR_CUDA, "cudaGetSymbolAddress", e);
    e = cudaDeviceGetAttribute(&g_na_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return na_fail(RT_ERR_CUDA, "device attribute", e);
    float4* tab = (float4*)((unsigned char*)p + kNaTabOff);
    for (int l = 0; l <= kNaTableLevels; ++l) {
      e = launch_direction_table(l, tab, 0);
      if (e != cudaSuccess) return na_fail(RT_ERR_CUDA, "direction table", e);
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return na_fail(RT_ERR_CUDA, "direction table", e);
    g_na_ptr[dev] = (unsigned char*)p;
  }
  *base = g_na_ptr[dev];
  *sms = g_na_sms[dev];
  return RT_OK;
}

bool na_exact(double v) { return v == ldexp(floor(ldexp(v, 4)), -4) && fabs(v) <= 4096.0; }

// The FP32 walker deposits Gamma in eV/s (an FP32 erg/s deposit of a faintly
// lit cell would fall below the FP32 normal range); the caller's array is
// turned into erg/s in place afterwards, the product taken in FP64 as
// rt_get_rates takes it.
__global__ void na_scale_kernel(float* a, long long n, double scale) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    a[c] = (float)((double)a[c] * scale);
}

}  // namespace

extern "C" {

const char* rt_noalloc_last_error(void) { return g_na_error.c_str(); }

int rt_trace_noalloc(const rt_noalloc_grid* g, int nsrc, const double* pos_cm, const double* ndot,
                     const double* e_ph_eV, const double* sigma_cm2, const rt_trace_params* p, void* stream,
                     rt_budget* out) {
  if (!g || !p || !out) return na_fail(RT_ERR_INVALID_ARG, "NULL argument");
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || (long long)g->nx * g->ny * g->nz >= (1LL << 31))
    return na_fail(RT_ERR_INVALID_ARG, "grid dimensions");
  if (!(g->box_len_cm > 0) || !isfinite(g->box_len_cm)) return na_fail(RT_ERR_INVALID_ARG, "box_len_cm");
  if (!g->n_HI || !g->n_H || !g->x_HI || !g->kph || !g->gamma)
    return na_fail(RT_ERR_INVALID_ARG, "every grid array is required");
  if (nsrc < 0 || nsrc > RT_NOALLOC_MAX_SOURCES)
    return na_fail(RT_ERR_INVALID_ARG, "more sources than RT_NOALLOC_MAX_SOURCES (1024)");
  if (nsrc > 0 && (!pos_cm || !ndot || !e_ph_eV || !sigma_cm2)) return na_fail(RT_ERR_INVALID_ARG, "source arrays");
  if (p->level0 < 0 || p->max_level < p->level0 || p->max_level > RT_MAX_LEVEL || !(p->phi_c > 0) ||
      !(p->f_term > 0 && p->f_term < 1) || p->segs_per_iter < 0 || p->segs_per_iter > 1024 ||
      p->blocks_per_sm < 0 || p->blocks_per_sm > 32 || p->passes < 0 || p->passes > 1 || p->light_cm != 0.0)
    return na_fail(RT_ERR_INVALID_ARG, "trace parameters");
  if (p->queue_capacity > RT_NOALLOC_MAX_RECORDS)
    return na_fail(RT_ERR_INVALID_ARG, "queue_capacity above RT_NOALLOC_MAX_RECORDS (262144)");
  const double dx = g->box_len_cm / g->nx;
  const double ext[3] = {g->nx * dx, g->ny * dx, g->nz * dx};
  for (int i = 0; i < nsrc; ++i) {
    for (int a = 0; a < 3; ++a)
      if (!(pos_cm[3 * i + a] >= 0 && pos_cm[3 * i + a] <= ext[a])) return na_fail(RT_ERR_INVALID_ARG, "source outside the box");
    if (!(ndot[i] >= 0) || !isfinite(ndot[i]) || !(e_ph_eV[i] >= kEHI) || !isfinite(e_ph_eV[i]) ||
        !(sigma_cm2[i] >= 0) || !isfinite(sigma_cm2[i]))
      return na_fail(RT_ERR_INVALID_ARG, "source parameters");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(RT_ERR_CUDA, "cudaGetDevice", e);
  unsigned char* base = nullptr;
  int sms = 0;
  int rc = na_setup(dev, &base, &sms);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* ctl = (unsigned long long*)(base + kNaCtlOff);
  double* acc = (double*)(base + kNaAccOff);
  unsigned long long* cnt = (unsigned long long*)(base + kNaCntOff);
  InstDev* inst = (InstDev*)(base + kNaInstOff);
  SourceDev* src = (SourceDev*)(base + kNaSrcOff);
  const size_t ncell = (size_t)g->nx * g->ny * g->nz;

  // Step 2: zero the outputs and the budget sums (no allocation: memsets)
  if ((e = cudaMemsetAsync(g->kph, 0, ncell * sizeof(float), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(g->gamma, 0, ncell * sizeof(float), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(acc, 0, kNaAccWords * sizeof(double), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(cnt, 0, kCntWords * sizeof(unsigned long long), st)) != cudaSuccess)
    return na_fail(RT_ERR_CUDA, "clearing outputs", e);

  // grid descriptor and source records, staged through small host buffers on
  // the stack (the stream is synchronised before they go out of scope)
  InstDev I;
  memset(&I, 0, sizeof I);
  I.nx = g->nx; I.ny = g->ny; I.nz = g->nz;
  I.nhi = g->n_HI; I.nH = g->n_H; I.xHI = g->x_HI; I.K = g->kph; I.G = g->gamma; I.acc = acc; I.cnt = cnt;
  if ((e = cudaMemcpyAsync(inst, &I, sizeof I, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return na_fail(RT_ERR_CUDA, "grid descriptor", e);
  const double npix0 = 12.0 * ldexp(1.0, 2 * p->level0);
  const double vol = dx * dx * dx;
  constexpr int kChunk = 32;
  SourceDev chunk[kChunk];
  for (int i0 = 0; i0 < nsrc; i0 += kChunk) {
    const int m = nsrc - i0 < kChunk ? nsrc - i0 : kChunk;
    for (int j = 0; j < m; ++j) {
      const int i = i0 + j;
      SourceDev& S = chunk[j];
      memset(&S, 0, sizeof S);
      for (int a = 0; a < 3; ++a) S.s[a] = pos_cm[3 * i + a] / dx;
      S.sdx = sigma_cm2[i] * dx;
      S.heat = (e_ph_eV[i] - kEHI) * kEvErg;
      S.unit = ndot[i] / npix0;
      S.w = S.unit * sigma_cm2[i] / (dx * dx);
      S.rw = S.unit / vol;
      S.inst = 0;
      S.local = i;
      int exact = 1;
      float s32[3], slo[3], sab[3];
      for (int a = 0; a < 3; ++a) {
        s32[a] = (float)S.s[a];
        slo[a] = (float)(S.s[a] - (double)s32[a]);
        sab[a] = ((double)s32[a] + (double)slo[a] == S.s[a]) ? 0.0f : (float)ldexp(fabs(S.s[a]), -46);
        exact &= na_exact(S.s[a]) ? 1 : 0;
      }
      S.exact32 = exact && g->nx <= 4096 && g->ny <= 4096 && g->nz <= 4096;
      S.k32 = make_float4((float)S.sdx, (float)S.w, (float)S.rw, (float)(e_ph_eV[i] - kEHI));  // heat in eV
      S.s32 = make_float4(s32[0], s32[1], s32[2], S.exact32 ? 1.0f : 0.0f);
      S.slo32 = make_float4(slo[0], slo[1], slo[2], (float)(S.sdx - (double)(float)S.sdx));
      S.sabs32 = make_float4(sab[0], sab[1], sab[2], 0.0f);
    }
    if ((e = cudaMemcpyAsync(src + i0, chunk, m * sizeof(SourceDev), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return na_fail(RT_ERR_CUDA, "source records", e);
  }

  const unsigned long long n_roots = (unsigned long long)npix0 * (unsigned long long)nsrc;
  if ((e = launch_trace_init(ctl, base + kNaQueueOff, kNaQueueBytes, n_roots, 1, FLIGHT_OFF, 0, 0, 1, st)) !=
      cudaSuccess)
    return na_fail(RT_ERR_CUDA, "trace init", e);
  if (n_roots > 0) {
    TraceArgs A;
    memset(&A, 0, sizeof A);
    A.inst = inst;
    A.ninst = 1;
    A.src = src;
    A.nsrc = nsrc;
    A.level0 = p->level0;
    A.max_level = p->max_level;
    A.npix0 = (uint32_t)npix0;
    A.n_roots = n_roots;
    for (int l = 0; l < kLevels; ++l) {
      A.rsplit[l] = sqrt((12.0 * ldexp(1.0, 2 * l)) / (4.0 * M_PI * p->phi_c));
      A.rsplit32[l] = (float)A.rsplit[l];
      A.rsplit32lo[l] = (float)(A.rsplit[l] - (double)A.rsplit32[l]);
    }
    A.dir_tab = (const float4*)(base + kNaTabOff);
    A.dir_levels = kNaTableLevels;
    A.tau_term = -log(p->f_term);
    A.tau_term32 = (float)A.tau_term;
    A.tau_term32lo = (float)(A.tau_term - (double)A.tau_term32);
    A.queue = base + kNaQueueOff;
    A.cap = p->queue_capacity > 0 ? (unsigned long long)p->queue_capacity : (unsigned long long)RT_NOALLOC_MAX_RECORDS;
    A.ctl = ctl;
    A.timeout_ns = (long long)((p->timeout_s > 0 ? p->timeout_s : 2.0) * 1e9);
    A.segs_per_iter = p->segs_per_iter > 0 ? p->segs_per_iter : 8;
    A.max_steps = 2 * (g->nx + g->ny + g->nz) + 16;
    A.checksums = (p->flags & RT_TRACE_CHECKSUMS) != 0;
    A.fc = (p->flags & RT_TRACE_FC) != 0;
    for (int l = 0; l < kLevels; ++l) {
      A.theta[l] = sqrt(4.0 * M_PI / (12.0 * ldexp(1.0, 2 * l)));
      A.theta32[l] = (float)A.theta[l];
    }
    int per_sm = 0;
    if ((e = trace_occupancy(RT_FP32_MIXED, 0, 256, &per_sm)) != cudaSuccess) return na_fail(RT_ERR_CUDA, "occupancy", e);
    if (per_sm < 1) per_sm = 1;
    if (p->blocks_per_sm > 0 && p->blocks_per_sm < per_sm) per_sm = p->blocks_per_sm;
    if (per_sm * sms > kNaMaxBlocks) return na_fail(RT_ERR_INVALID_ARG, "more trace blocks than the budget rows hold");
    A.blk = (double*)(base + kNaBlkOff);
    A.blk_rows = 1;
    if ((e = launch_trace(RT_FP32_MIXED, 0, A, per_sm * sms, 256, st)) != cudaSuccess)
      return na_fail(RT_ERR_CUDA, "trace launch", e);
    long long blocks = ((long long)ncell + 255) / 256;
    if (blocks > 8LL * sms) blocks = 8LL * sms;
    na_scale_kernel<<<(int)blocks, 256, 0, st>>>(g->gamma, (long long)ncell, kEvErg);
    if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(RT_ERR_CUDA, "Gamma to erg/s", e);
  }
  // result: budget, counters and control words
  double hacc[4];
  unsigned long long hcnt[kCntWords], hctl[CTL_N];
  if ((e = cudaMemcpyAsync(hacc, acc, sizeof hacc, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(hcnt, cnt, sizeof hcnt, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(hctl, ctl, sizeof hctl, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return na_fail(RT_ERR_CUDA, "reading the budget", e);
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
  out->queue_pushed = hctl[CTL_TAIL];
  out->status = (int)hctl[CTL_STATUS];
  if (out->status == RT_ERR_QUEUE_OVERFLOW)
    return na_fail(RT_ERR_QUEUE_OVERFLOW, "the trace needs more than RT_NOALLOC_MAX_RECORDS (262144) queue records");
  if (out->status != RT_OK) return na_fail(out->status, "device status");
  g_na_error.clear();
  return RT_OK;
}

}  // extern "C"
