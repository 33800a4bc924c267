// rt_internal.cuh -- device-side data layout and helpers shared by the
// library's kernels (trace.cu, chem.cu) and its host code (api.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt.h"

namespace rtg {

constexpr int kLevels = RT_MAX_LEVEL + 1;
constexpr double kEvErg = 1.602176634e-12;  // erg per eV
constexpr double kEHI = 13.6;               // hydrogen threshold, eV (Sec. 2.2)
// Photon types (Sec. 3.2): 0 ionises H I, 1 He I, 2 He II; each is absorbed
// by its own species, with these ionisation energies (eV)
constexpr int kTypes = 3;
constexpr double kEIon[kTypes] = {13.6, 24.6, 54.4};

// Control words of one trace (64-bit each), in device memory.  The three
// that every warp updates or polls sit in cache lines of their own, so their
// atomics and loads do not queue behind one another in L2.
enum CtlWord {
  CTL_HEAD = 0,          // next ticket to hand out
  CTL_TAIL = 16,         // queue slots reserved by producers
  CTL_OUTSTANDING = 32,  // live packages (signed)
  CTL_STATUS = 48,       // RT_OK or first device error (atomicCAS)
  CTL_EPOCH = 49,        // tag of this trace's queue records
  CTL_PEAK = 50,         // largest TAIL of the earlier passes of this trace
  CTL_PUSHED = 51,       // sum of TAIL over the earlier passes of this trace
  CTL_RESUME = 52,       // packages in flight from the previous trace (input store)
  CTL_RES_A = 53,        // this pass continues input records [RES_A, RES_B)
  CTL_RES_B = 54,
  CTL_HALTED = 56,       // packages halted so far in this trace (output store slots)
  CTL_SET_ERR = 57,      // RT_ERR_INVALID_ARG once an asynchronously uploaded state was
                         // rejected (until the host reports it); copied into STATUS
                         // by every trace
  CTL_SET_BADN = 58,     // first rejected cell of that state: n_H, x_HI (~0 = none)
  CTL_SET_BADX = 59,
  CTL_CHECK_N = 60,      // scratch of the state check: first bad n_H cell, x_HI cell
  CTL_CHECK_X = 61,
  CTL_INIT_DONE = 62,    // blocks of the queue reset that have finished (reset to 0 by the last)
  CTL_COMMIT_DONE = 63,  // blocks of a state commit that have finished (reset to 0 by the last)
  CTL_N = 64             // words (512 bytes)
};

// trace_init_kernel modes for the in-flight stores (finite speed of light)
enum FlightMode {
  FLIGHT_OFF = 0,      // nothing in flight: RESUME = HALTED = 0
  FLIGHT_ADVANCE = 1,  // a new trace continues what the previous one halted
  FLIGHT_RETRY = 2     // the same trace again (after growing a store): keep RESUME
};

// One point source, prepared on the host for the kernels.  P of a package is
// carried in units of the root package's photon rate (root P = 1 exactly),
// so every per-source constant below folds in unit = ndot / npix0.
struct __align__(16) SourceDev {
  // FP32 view (mixed path), one 16-byte load each
  float4 k32;     // sdx, w, rw, heat (see the FP64 fields)
  float4 s32;     // position as FP32 pair, high part; .w = 1 if exact32
  float4 slo32;   // low part (s - s32); .w = sdx - k32.x
  float4 sabs32;  // 2^-46 |s| where the pair does not hold s exactly, else 0; .w = p0
  // FP64 view
  double s[3];    // position in cell units (pos_cm / dx)
  double sdx;     // sigma * dx: optical depth per unit n_HI per cell length
  double w;       // unit * sigma / dx^2: k_ph per unit P per cell length (phi = 1)
  double rw;      // unit / dx^3: k_ph per unit P per unit n_HI (residual absorption)
  double heat;    // (E_ph - 13.6 eV) in erg
  double unit;    // photons/s carried by P = 1
  double p0;      // P of a new package (finite speed of light; sabs32.w in FP32):
                  // 1, unless the unit is kept for packages still in flight
                  // while the source's rate has changed
  int inst;       // owning grid slot
  int local;      // index of the source within its grid (checksum)
  int exact32;    // position on a 1/16-cell lattice within 4096 cells (see api.cu)
  int type;       // photon type of its packages (0 H I, 1 He I, 2 He II)
};

// InstDev.flags: the FP32-mixed grid stores n_HI as float2 pairs (n_HI
// rounded to FP32, and the remainder), so the walker sums optical depth to
// ~2^-44 of the FP64 evaluation.
constexpr int kInstNhiPair = 1;

// One grid (instance) as the trace kernel sees it.
struct InstDev {
  int nx, ny, nz;
  int flags;                // kInstNhiPair: nhi holds (hi, lo) FP32 pairs
  const void* nhi;          // absorber density n_HI (double, float or float2), x fastest
  const double* nH;         // hydrogen density, FP64 (decisions re-taken in FP64)
  const double* xHI;        // neutral fraction, FP64
  double* xHII;             // ionised fraction, FP64 (chemistry)
  void* K;                  // k_ph accumulator (double or float)
  void* G;                  // Gamma accumulator (double or float)
  double* acc;              // [0] emitted [1] absorbed [2] escaped [3] resumed [4] halted (photons/s)
  unsigned long long* cnt;  // [0,15) counts, [15,30) hashes, [30] segments, [31], [32] fallbacks
  // helium photon types 1, 2 (null until the grid has helium absorbers):
  const void* nhe[2];       // absorber density as nhi (FP64, or FP32 pairs)
  const double* nhe64[2];   // the same in FP64 (decisions re-taken in FP64)
  void* Khe[2];             // their k_ph and Gamma accumulators
  void* Ghe[2];
};
constexpr int kCntSegments = 2 * kLevels;
constexpr int kCntFallbacks = 2 * kLevels + 1;
constexpr int kCntFallbacksTau = 2 * kLevels + 2;
constexpr int kCntWords = 2 * kLevels + 3;

// Per-block budget rows of a trace launch (global memory, one buffer per
// grid or batch): for each block and each of the launch's first kBlkGrids
// grids, kBlkRow 8-byte words (emitted, absorbed, escaped, resumed, halted
// as doubles, then the segment count as an unsigned 64-bit integer).  A
// lane adds its sums there with fire-and-forget reductions when its next
// package belongs to another grid; the block adds its rows into the grid's
// sums when it finishes.
constexpr int kBlkGrids = 64;
constexpr int kBlkRow = 6;
constexpr int kBlkMaxPerSM = 8;  // 256-thread blocks: at most 2048 threads per SM
inline size_t blk_rows_bytes(int num_sms, int rows) {
  return (size_t)num_sms * kBlkMaxPerSM * (size_t)rows * kBlkRow * sizeof(double);
}

// Queue records.  The tag word is written last with release semantics and
// equals the trace's epoch once the record is complete.  The same layouts
// hold packages in flight between traces (finite speed of light), where the
// tag is not used as one.
struct __align__(16) Rec64 {
  double r, P, tau;
  uint32_t src, pix;
  uint32_t level;  // level | age << 4
  uint32_t tag;    // epoch; in flight: the cell index
};
struct __align__(16) Rec32 {
  float r, r_lo;  // radius as an FP32 pair
  float P, tau;   // photon rate; optical depth as an FP32 pair (tau, tau_lo)
  float tau_lo;
  float tau_err;  // bound on |tau (pair) - tau (FP64 evaluation)|
  uint32_t src, pix;
  uint32_t tag;   // (epoch << 4) | level
  uint32_t age;   // traces since emission (finite speed of light)
  uint32_t cell;  // in flight: the cell index
  uint32_t pad;
};
// Queue record of the FP32-mixed walker when packages do not outlive the
// trace (no finite speed of light): one 32-byte sector.  The level rides in
// the top 4 bits of the source index, and the tag word holds the low 16 bits
// of the trace epoch above the error bound tau_err rounded up to bf16 (a
// wider bound only sends more decisions to FP64).  Epochs whose low 16 bits
// are 0 are never used, and the queue is cleared before the epoch that would
// repeat them (trace_init_kernel), so zeroed or stale slots never match.
struct __align__(32) QRec32 {
  float r, r_lo, P, tau;
  float tau_lo;
  uint32_t src_lv;  // src | level << 28
  uint32_t pix;
  uint32_t tag;     // (epoch & 0xffff) << 16 | bf16(tau_err)
};
constexpr unsigned long long kEpochMask = 0xffffULL;
constexpr uint32_t kMaxQueueSources = 1u << 28;  // source indices of QRec32
static_assert(sizeof(Rec64) == 48, "record layout");
static_assert(sizeof(Rec32) == 48, "record layout");
static_assert(sizeof(QRec32) == 32, "record layout");
static_assert(RT_MAX_LEVEL < 16, "the level takes 4 bits of a queue record");

// Bytes of one queue record of a trace.
inline size_t queue_rec_bytes(int fp64, bool fsl) {
  return fp64 ? sizeof(Rec64) : fsl ? sizeof(Rec32) : sizeof(QRec32);
}

struct TraceArgs {
  const InstDev* inst;
  int ninst;
  const SourceDev* src;     // every source of the launch (packages name them by index)
  int nsrc;
  int src_first;            // this pass emits sources [src_first, src_first + n_roots / npix0)
  int level0, max_level;
  uint32_t npix0;
  unsigned long long n_roots;
  double rsplit[kLevels];
  float rsplit32[kLevels];    // R_split as the FP32 pair (rsplit32, rsplit32lo)
  float rsplit32lo[kLevels];
  const float4* dir_tab;      // pixel directions as FP32 pairs, levels 0..dir_levels
  int dir_levels;             // -1: no table
  double tau_term;
  float tau_term32, tau_term32lo;  // tau_term as an FP32 pair
  void* queue;
  unsigned long long cap;
  unsigned long long* ctl;
  long long timeout_ns;
  int segs_per_iter;
  int max_steps;  // bound on segments of one package (guards the DDA loop)
  int checksums;  // accumulate the created-set checksum
  int fc;         // scale k_ph and Gamma deposits by the covering factor (Eq. "fc")
  double theta[kLevels];    // pixel width sqrt(4 pi / N_pix(l)) in radians
  float theta32[kLevels];
  // finite speed of light (the kernel instantiated for it reads these)
  const double* rlim64;     // halting radius per age, cell units
  const float2* rlim32;     // the same as FP32 pairs
  int n_ages;
  const void* res_in;       // packages halted by the previous trace (Rec)
  void* halt_out;           // packages this trace halts (Rec)
  unsigned long long halt_cap;
  // per-block budget rows: [gridDim.x][blk_rows][kBlkRow] words,
  // blk_rows = min(ninst, kBlkGrids); each block clears its own rows
  double* blk;
  int blk_rows;
};

// 64-bit finaliser used for the created-package checksum (documented in rt.h).
__host__ __device__ __forceinline__ uint64_t pkg_hash(uint32_t src, uint32_t level, uint64_t pix) {
  uint64_t x = ((uint64_t)src << 40) ^ ((uint64_t)level << 34) ^ pix;
  x ^= x >> 31;
  x *= 0x7fb5d329728ea185ULL;
  x ^= x >> 27;
  x *= 0x81dadef4bc2dd44dULL;
  x ^= x >> 33;
  return x;
}

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ long long ld_acquire_s64(const unsigned long long* p) {
  long long v;
  asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void set_status(unsigned long long* ctl, int code) {
  atomicCAS(&ctl[CTL_STATUS], 0ULL, (unsigned long long)code);
}
#endif

}  // namespace rtg
