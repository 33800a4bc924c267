// trace.cu -- persistent ray-tracing kernel (Sec. 2.1-2.2, Steps 1-5 of
// Sec. 3.1) for one or many grids at once.
//
// Work model.  Every lane of the persistent grid carries at most one photon
// package.  A lane without a package takes a ticket from a global counter
// (one atomic per warp).  Tickets below n_roots are root packages (Step 1:
// source = ticket / N_pix, pixel = ticket % N_pix, P = 1 in units of the
// source's Ndot / N_pix) and need no memory; higher tickets name queue slots
// that split packages publish.  When a package splits (Step 3e) its lane
// keeps child 0 and hands children 1-3 to lanes of its warp whose package
// ended in the same round (no package, no ticket), by warp shuffles; the
// rest go to the queue (one atomic per warp reserves the slots), where each
// 32-byte record's tag word is stored last with release semantics and
// polled with acquire loads.  An outstanding-package counter
// (+3 per split, -1 per finished package) tells idle warps when the trace is
// over.  Every wait is bounded: a warp that sees no change of the counter for
// timeout_ns sets RT_ERR_TIMEOUT and leaves; a package that takes more steps
// than a ray can cross planes sets RT_ERR_STATE.  Nothing traps.
//
// Per segment (Steps 3d-3i): next crossing r_next = min_i t_i (Eq. "trace"),
// split test r_next > R_split(l) (Eq. "split"), tau = sigma n_HI dr
// (Eq. "dtau"), dP = P (1 - e^-tau) (Eq. "flux"), k_ph += P w dr phi(tau)
// with phi = (1 - e^-tau)/tau (Eq. "kph"), Gamma += k_ph (E - 13.6 eV)
// (Eq. "gamma"), then termination at tau_tot > -ln f_term with the residual
// absorbed in place, and exit at the box boundary.
//
// Finite speed of light (Step 3j; the kernel instantiated with FSL): a
// package of age a (traces since its emission) halts where its crossing
// radius would pass rlim[a]; the cut segment is deposited, the termination
// test comes first, and the package is appended to an output store with its
// cell.  The next trace's tickets n_roots .. n_roots + n_res - 1 name the
// stored packages, which continue from their cells.  This instantiation
// queues every child 1-3, in 48-byte records that carry the age.
#include <type_traits>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "f2.cuh"
#include "healpix.cuh"
#include "rt_internal.cuh"

#ifndef TRACE_MIN_BLOCKS
#define TRACE_MIN_BLOCKS 2
#endif

namespace rtg {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kShInst = 64;  // grids whose level counters and fallback counts a block keeps in shared memory
static_assert(kBlkGrids <= kShInst, "a grid with a budget row has its counters in shared memory");
constexpr int kBlock = 256;  // threads per block of the trace kernel

enum Event { EV_NONE = 0, EV_SPLIT = 1, EV_DONE = 2, EV_HALT = 3 };
constexpr int kAcc = 5;  // budget sums per grid: emitted, absorbed, escaped, resumed, halted

// Photon budget of one lane for the grid it is working on; lives in shared
// memory (one slot per thread) and is touched only at package events.
// Position of the set bit of rank n (0 = lowest) in m; m holds more than n
// set bits.  A binary search on the population counts of the low halves.
__device__ __forceinline__ int nth_set_bit(unsigned m, unsigned n) {
  int pos = 0;
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) {
    const unsigned low = m & ((1u << w) - 1u);
    const unsigned c = (unsigned)__popc(low);
    if (c <= n) {
      n -= c;
      m >>= w;
      pos += w;
    } else {
      m = low;
    }
  }
  return pos;
}

struct LaneAcc {
  double emitted, absorbed, escaped, resumed, halted;
  unsigned long long segments;
  unsigned int fallbacks, fallbacks_tau;
  int inst;
  // 72 bytes = 18 banks: the 8-byte accesses of a half-warp to one field
  // fall on 16 different bank pairs (a 64-byte stride puts them on two)
  unsigned int pad[3];
};
static_assert(sizeof(LaneAcc) == 72, "conflict-free stride of the per-lane sums");

// A block's budget sums per grid for the first kBlkGrids grids of the
// launch: its rows of TraceArgs.blk (global memory, kBlkRow words per grid)
// and, for the rare fallback counts, a table in shared memory.  A lane that
// moves to a package of another grid adds its sums to the rows with
// reductions whose results it does not wait for; the block adds its rows
// into the grids' sums once at the end.  (Shared-memory FP64 atomics, which
// return their result, cost the 64-grid batch 11 % of its trace time.)
struct BlockBudget {
  double* rows;             // [nrows][kBlkRow]: emitted, absorbed, escaped, resumed, halted, segments
  int nrows;                // min(grids of the launch, kBlkGrids)
  unsigned int* fb;         // [kShInst][2]: fallbacks, fallbacks_tau
};

// Grids beyond the block's rows (rare: batches of more than kBlkGrids
// grids) flush to the grid's sums directly, out of line.
__device__ __noinline__ void acc_flush_global(const LaneAcc& a, const TraceArgs& A) {
  const InstDev& I = A.inst[a.inst];
  if (a.emitted != 0.0) atomicAdd(&I.acc[0], a.emitted);
  if (a.absorbed != 0.0) atomicAdd(&I.acc[1], a.absorbed);
  if (a.escaped != 0.0) atomicAdd(&I.acc[2], a.escaped);
  if (a.resumed != 0.0) atomicAdd(&I.acc[3], a.resumed);
  if (a.halted != 0.0) atomicAdd(&I.acc[4], a.halted);
  if (a.segments) atomicAdd(&I.cnt[kCntSegments], a.segments);
  if (a.fallbacks) atomicAdd(&I.cnt[kCntFallbacks], (unsigned long long)a.fallbacks);
  if (a.fallbacks_tau) atomicAdd(&I.cnt[kCntFallbacksTau], (unsigned long long)a.fallbacks_tau);
}
__device__ __forceinline__ void acc_flush(LaneAcc& a, const TraceArgs& A, const BlockBudget& bb) {
  if (a.inst >= 0 && a.inst < bb.nrows) {
    // straight-line reductions (adding zeros costs less than branching)
    double* t = bb.rows + kBlkRow * a.inst;
    atomicAdd(&t[0], a.emitted);
    atomicAdd(&t[1], a.absorbed);
    atomicAdd(&t[2], a.escaped);
    if (a.resumed != 0.0 || a.halted != 0.0) {
      atomicAdd(&t[3], a.resumed);
      atomicAdd(&t[4], a.halted);
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(&t[kAcc]), a.segments);
    if (a.fallbacks | a.fallbacks_tau) {
      atomicAdd(&bb.fb[2 * a.inst], a.fallbacks);
      atomicAdd(&bb.fb[2 * a.inst + 1], a.fallbacks_tau);
    }
  } else if (a.inst >= 0) {
    acc_flush_global(a, A);
  }
  a.emitted = a.absorbed = a.escaped = a.resumed = a.halted = 0.0;
  a.segments = 0;
  a.fallbacks = 0;
  a.fallbacks_tau = 0;
}

// Switch the lane's budget to grid `inst`, flushing the previous grid's sums
// (with the segments counted since the last switch).
__device__ __forceinline__ void acc_switch(LaneAcc& a, unsigned& nseg, int inst, const TraceArgs& A,
                                           const BlockBudget& bb) {
  if (a.inst != inst) {
    a.segments += nseg;
    nseg = 0;
    acc_flush(a, A, bb);
    a.inst = inst;
  }
}

struct LevelCounters {
  unsigned int* cnt;        // [kShInst][kLevels]
  unsigned long long* hsh;  // [kShInst][kLevels]
  // Count n packages (level, pix0 .. pix0 + n - 1) of a source; the
  // checksum terms only when requested.
  __device__ __forceinline__ void add(const TraceArgs& A, int inst, int local, int level, uint32_t pix0,
                                      uint32_t n) {
    unsigned long long h = 0;
    if (A.checksums)
      for (uint32_t k = 0; k < n; ++k) h += pkg_hash((uint32_t)local, (uint32_t)level, pix0 + k);
    if (inst < kShInst) {
      atomicAdd(&cnt[inst * kLevels + level], n);
      if (A.checksums) atomicAdd(&hsh[inst * kLevels + level], h);
    } else {
      atomicAdd(&A.inst[inst].cnt[level], (unsigned long long)n);
      if (A.checksums) atomicAdd(&A.inst[inst].cnt[kLevels + level], h);
    }
  }
};

// ---------------------------------------------------------------------------
// FP64 walker: every decision (cell of a point, next crossing, split,
// termination) is evaluated with explicitly rounded FP64 operations in the
// order a plain FP64 evaluation of the method's formulas uses.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_of64(double u, double n) {
  if (n > 0) return (int)floor(u);
  if (n < 0) return (int)ceil(u) - 1;
  return (int)floor(u);
}
__device__ __forceinline__ double next_t64(int c, double s, double n) {
  if (n > 0) return __ddiv_rn(__dsub_rn((double)(c + 1), s), n);
  if (n < 0) return __ddiv_rn(__dsub_rn((double)c, s), n);
  return __longlong_as_double(0x7ff0000000000000LL);  // +inf
}

struct Walk64 {
  using Rec = Rec64;
  template <bool FSL> using Q = Rec64;  // queue record
  uint32_t src, level, pix;
  uint32_t age;   // traces since emission (finite speed of light)
  double r, P, tau, Pstart;
  double rlim;    // halting radius of this age
  double s0, s1, s2, n0, n1, n2, t0, t1, t2;
  int c0, c1, c2;
  int nx, ny, nz, steps;
  unsigned nseg;
  const double* nhi;
  double* K;
  double* G;
  double sdx, w, rw, heat;

  __device__ __forceinline__ bool inside() const {
    return c0 >= 0 && c0 < nx && c1 >= 0 && c1 < ny && c2 >= 0 && c2 < nz;
  }
  __device__ __forceinline__ int inst(const TraceArgs& A) const { return A.src[src].inst; }
  __device__ __forceinline__ double unit(const TraceArgs& A) const { return A.src[src].unit; }
  __device__ __forceinline__ int lvl() const { return (int)level; }
  // P of a new package of source S (finite speed of light)
  __device__ __forceinline__ double emit(const SourceDev& S) {
    P = S.p0;
    return P;
  }

  __device__ __forceinline__ void bind(const TraceArgs& A) {
    const SourceDev& S = A.src[src];
    s0 = S.s[0]; s1 = S.s[1]; s2 = S.s[2];
    sdx = S.sdx; w = S.w; rw = S.rw; heat = S.heat;
    const InstDev& I = A.inst[S.inst];
    nx = I.nx; ny = I.ny; nz = I.nz;
    // the absorber and accumulators of the package's photon type (Sec. 3.2)
    const int t = S.type;
    nhi = (const double*)(t == 0 ? I.nhi : I.nhe[t - 1]);
    K = (double*)(t == 0 ? I.K : I.Khe[t - 1]);
    G = (double*)(t == 0 ? I.G : I.Ghe[t - 1]);
    double n[3];
    pix2vec64((int)level, pix, n);
    n0 = n[0]; n1 = n[1]; n2 = n[2];
    Pstart = P;
    steps = 0;
  }
  // Steps 3a-3b: direction and cell at radius r.  Returns false if the
  // package starts outside the box.
  __device__ __forceinline__ bool start(const TraceArgs& A) {
    bind(A);
    c0 = cell_of64(__dadd_rn(s0, __dmul_rn(r, n0)), n0);
    c1 = cell_of64(__dadd_rn(s1, __dmul_rn(r, n1)), n1);
    c2 = cell_of64(__dadd_rn(s2, __dmul_rn(r, n2)), n2);
    if (!inside()) return false;
    t0 = next_t64(c0, s0, n0);
    t1 = next_t64(c1, s1, n1);
    t2 = next_t64(c2, s2, n2);
    return true;
  }
  // A package continued from the previous trace: the cell it halted in.
  __device__ __forceinline__ void resume(const TraceArgs& A, uint32_t cell) {
    bind(A);
    c0 = (int)(cell % (uint32_t)nx);
    c1 = (int)((cell / (uint32_t)nx) % (uint32_t)ny);
    c2 = (int)(cell / ((uint32_t)nx * (uint32_t)ny));
    t0 = next_t64(c0, s0, n0);
    t1 = next_t64(c1, s1, n1);
    t2 = next_t64(c2, s2, n2);
  }
  __device__ __forceinline__ void set_rlim(const TraceArgs& A) {
    if ((int)age < A.n_ages) rlim = A.rlim64[age];
    else { set_status(A.ctl, RT_ERR_STATE); rlim = 0.0; }
  }

  __device__ __forceinline__ void load(const Rec& q) {
    r = q.r; P = q.P; tau = q.tau; src = q.src; pix = q.pix; level = q.level & 15u; age = q.level >> 4;
  }
  // Record of child cpix (level + 1, P/4, same radius, optical depth and age).
  __device__ __forceinline__ Rec make_child(uint32_t cpix) const {
    Rec c;
    c.r = r; c.P = P * 0.25; c.tau = tau; c.src = src; c.pix = cpix; c.level = (level + 1) | (age << 4); c.tag = 0;
    return c;
  }
  __device__ __forceinline__ static uint32_t cell_of_record(const Rec& q) { return q.tag; }
  // A halted package as the next trace continues it (one trace older).
  __device__ __forceinline__ void store_halted(Rec* q) const {
    Rec c;
    c.r = r; c.P = P; c.tau = tau; c.src = src; c.pix = pix; c.level = level | ((age + 1) << 4);
    c.tag = (uint32_t)(c0 + nx * (c1 + ny * c2));
    *q = c;
  }
  // Publish a record in the global queue: payload first, then the tag with
  // release semantics.  (The age travels in the level word either way.)
  template <bool FSL>
  __device__ __forceinline__ static void publish(Rec* q, const Rec& c, uint32_t epoch) {
    __stcg(reinterpret_cast<double2*>(&q->r), make_double2(c.r, c.P));
    __stcg(reinterpret_cast<double*>(&q->tau), c.tau);
    __stcg(reinterpret_cast<uint2*>(&q->src), make_uint2(c.src, c.pix));
    __stcg(&q->level, c.level);
    st_release_u32(&q->tag, epoch);
  }
  // Poll with an acquire load of the tag: the payload reads that follow a
  // successful poll are ordered after it without a fence.
  template <bool FSL>
  __device__ __forceinline__ static bool poll(const Rec* q, uint32_t epoch, Rec& o) {
    if (ld_acquire_u32(&q->tag) != epoch) return false;
    const double2 a = __ldcg(reinterpret_cast<const double2*>(&q->r));    // r, P
    const double2 b = __ldcg(reinterpret_cast<const double2*>(&q->tau));  // tau, (src, pix)
    const uint2 c = __ldcg(reinterpret_cast<const uint2*>(&q->level));    // level, tag
    const unsigned long long sp = (unsigned long long)__double_as_longlong(b.y);
    o.r = a.x; o.P = a.y; o.tau = b.x;
    o.src = (uint32_t)(sp & 0xffffffffu);
    o.pix = (uint32_t)(sp >> 32);
    o.level = c.x;
    return true;
  }
  // Every lane takes the record that lane `from` holds (all lanes call it).
  __device__ __forceinline__ static void shfl_rec(Rec& c, int from) {
    c.r = __shfl_sync(0xffffffffu, c.r, from);
    c.P = __shfl_sync(0xffffffffu, c.P, from);
    c.tau = __shfl_sync(0xffffffffu, c.tau, from);
    c.src = __shfl_sync(0xffffffffu, c.src, from);
    c.pix = __shfl_sync(0xffffffffu, c.pix, from);
    c.level = __shfl_sync(0xffffffffu, c.level, from);
  }
  __device__ __forceinline__ static Rec root_rec(uint32_t gsrc, uint32_t lvl0, uint32_t p) {
    Rec c;
    c.r = 0.0; c.P = 1.0; c.tau = 0.0; c.src = gsrc; c.pix = p; c.level = lvl0; c.tag = 0;
    return c;
  }
  __device__ __forceinline__ void become_child0() {
    level += 1; pix = 4u * pix; P = P * 0.25;
  }

  // One segment.  Returns EV_SPLIT before traversing a cell whose exit radius
  // exceeds R_split, EV_DONE when the package is absorbed or leaves the box,
  // EV_HALT (FSL) when it has travelled to its halting radius.
  template <bool FSL>
  __device__ __forceinline__ int step(const TraceArgs& A, LaneAcc& acc) {
    const double rn = fmin(t0, fmin(t1, t2));
    if ((int)level < A.max_level && rn > A.rsplit[level]) return EV_SPLIT;
    const bool halt = FSL && rn > rlim;  // Step 3j
    double dr = __dsub_rn(halt ? rlim : rn, r);
    if (dr < 0) dr = 0;
    const int idx = c0 + nx * (c1 + ny * c2);
    const double nh = __ldg(&nhi[idx]);
    const double dtau = __dmul_rn(__dmul_rn(sdx, nh), dr);
    const double am = -expm1(-dtau);
    const double phi = dtau > 0 ? am / dtau : 1.0;
    // covering factor (Eq. "fc"): pixel width at r, midpoint to nearest face
    double fcv = 1.0;
    if (A.fc) {
      const double L = r * A.theta[level];
      if (L > 0.0) {
        const double rm = r + 0.5 * dr;
        const double d = fmax(fabs(s0 + n0 * rm - (c0 + 0.5)),
                              fmax(fabs(s1 + n1 * rm - (c1 + 0.5)), fabs(s2 + n2 * rm - (c2 + 0.5))));
        const double f = 0.5 + (0.5 - d) / L;
        fcv = fmin(1.0, f * f);
      }
    }
    const double kadd = P * w * dr * phi * fcv;
    atomicAdd(&K[idx], kadd);
    if (heat != 0.0) atomicAdd(&G[idx], kadd * heat);
    if (dr > 0) nseg++;
    P = P - P * am;
    tau = __dadd_rn(tau, dtau);
    if (tau > A.tau_term) {
      const double kres = P * rw / nh * fcv;
      atomicAdd(&K[idx], kres);
      if (heat != 0.0) atomicAdd(&G[idx], kres * heat);
      acc.absorbed += Pstart * unit(A);
      return EV_DONE;
    }
    if (halt) {
      r = rlim;
      const double u = unit(A);
      acc.absorbed += (Pstart - P) * u;
      acc.halted += P * u;
      return EV_HALT;
    }
    if (n0 != 0 && t0 == rn) { c0 += n0 > 0 ? 1 : -1; t0 = next_t64(c0, s0, n0); }
    if (n1 != 0 && t1 == rn) { c1 += n1 > 0 ? 1 : -1; t1 = next_t64(c1, s1, n1); }
    if (n2 != 0 && t2 == rn) { c2 += n2 > 0 ? 1 : -1; t2 = next_t64(c2, s2, n2); }
    r = rn;
    if (!inside()) {
      const double u = unit(A);
      acc.absorbed += (Pstart - P) * u;
      acc.escaped += P * u;
      return EV_DONE;
    }
    if (++steps > A.max_steps) {
      set_status(A.ctl, RT_ERR_STATE);
      const double u = unit(A);
      acc.absorbed += (Pstart - P) * u;
      acc.escaped += P * u;
      return EV_DONE;
    }
    return EV_NONE;
  }
  // Budget of the parent's run when it splits (children carry P/4 each).
  __device__ __forceinline__ void on_split(const TraceArgs& A, LaneAcc& acc) const {
    acc.absorbed += (Pstart - P) * unit(A);
  }
  __device__ __forceinline__ void on_start_outside(const TraceArgs& A, LaneAcc& acc) const {
    acc.escaped += P * unit(A);
  }
};

// Optical depth that the FP64 evaluation accumulates along the lineage of
// package (level, pix) of source src up to and including its segment in cell
// (tc0, tc1, tc2).  Follows the FP64 path from the root: the root pixel at
// level0 is pix >> 2 (level - level0); at each split the lineage continues
// with the child on the path to pix.  If the lineage does not
// reach that cell at that level (returns NaN; the caller then keeps its FP32
// decision).  Takes values only, like decide64.
__device__ __noinline__ double retrace_tau64(const TraceArgs& A, uint32_t src, int level, uint32_t pix, int tc0,
                                             int tc1, int tc2) {
  const SourceDev& S = A.src[src];
  const InstDev& I = A.inst[S.inst];
  const double s0 = S.s[0], s1 = S.s[1], s2 = S.s[2];
  int l = A.level0;
  double r = 0.0, tau = 0.0;
  for (int guard = 0; guard <= RT_MAX_LEVEL + 1; ++guard) {
    const uint32_t p = pix >> (2 * (level - l));
    double n[3];
    pix2vec64(l, p, n);
    int c0 = cell_of64(__dadd_rn(s0, __dmul_rn(r, n[0])), n[0]);
    int c1 = cell_of64(__dadd_rn(s1, __dmul_rn(r, n[1])), n[1]);
    int c2 = cell_of64(__dadd_rn(s2, __dmul_rn(r, n[2])), n[2]);
    double t0 = next_t64(c0, s0, n[0]), t1 = next_t64(c1, s1, n[1]), t2 = next_t64(c2, s2, n[2]);
    bool split = false;
    for (int st = 0; st < A.max_steps; ++st) {
      if (c0 < 0 || c0 >= I.nx || c1 < 0 || c1 >= I.ny || c2 < 0 || c2 >= I.nz) return nan("");
      const double rn = fmin(t0, fmin(t1, t2));
      if (l < A.max_level && rn > A.rsplit[l]) { split = true; break; }
      double dr = __dsub_rn(rn, r);
      if (dr < 0) dr = 0;
      const int idx = c0 + I.nx * (c1 + I.ny * c2);
      const double nh = S.type == 0 ? __dmul_rn(I.nH[idx], I.xHI[idx]) : I.nhe64[S.type - 1][idx];
      tau = __dadd_rn(tau, __dmul_rn(__dmul_rn(S.sdx, nh), dr));
      if (l == level && c0 == tc0 && c1 == tc1 && c2 == tc2) return tau;
      if (tau > A.tau_term) return nan("");
      if (n[0] != 0 && t0 == rn) { c0 += n[0] > 0 ? 1 : -1; t0 = next_t64(c0, s0, n[0]); }
      if (n[1] != 0 && t1 == rn) { c1 += n[1] > 0 ? 1 : -1; t1 = next_t64(c1, s1, n[1]); }
      if (n[2] != 0 && t2 == rn) { c2 += n[2] > 0 ? 1 : -1; t2 = next_t64(c2, s2, n[2]); }
      r = rn;
    }
    if (!split || l >= level) return nan("");
    ++l;
  }
  return nan("");
}

// ---------------------------------------------------------------------------
// FP32-mixed walker.
//
// All per-segment arithmetic is FP32.  Crossing distances t_i, the radius r
// and segment lengths are carried as unevaluated FP32 pairs (hi + lo,
// "double-float"), built from the pixel direction stored as an FP32 pair
// (FP64 direction rounded twice) and from the source position as an FP32
// pair, so each t carries ~44 correct bits while every instruction is FP32.
// Optical depth, attenuation and the k_ph / Gamma deposits are plain FP32.
//
// Each decision that shapes the ray tree -- which cell plane is crossed next,
// whether the package splits, whether it terminates -- is taken from the
// FP32 values only when an error bound proves it equals the FP64 decision:
//   |t_pair - t_FP64| <= 2^-40 t + 2^-46 |s| / |n|   (per axis),
//   |tau_FP32 - tau_FP64| <= tau_err (accumulated per segment).
// Inside a band the decision is re-taken in FP64: the crossing distances of
// the current cell from the FP64 direction, or the FP64 optical depth of the
// package's lineage.  Per-level counts therefore equal the FP64 path's.
// ---------------------------------------------------------------------------
constexpr float kEps32 = 5.9604645e-8f;   // 2^-24
constexpr float kBandT = 9.094947e-13f;   // 2^-40
constexpr float kClose = 4.76837158e-7f;  // 2^-21: high parts farther apart are ordered

// Direction of (level, pix) as FP32 pairs: from the device table when the
// level is tabulated, else from the FP64 evaluation.  Returns the
// 45-degree-meridian flag.
__device__ __forceinline__ int dir_pair(const TraceArgs& A, int level, uint32_t pix, F2 n[3]) {
  if (level <= A.dir_levels) {
    const size_t idx = (size_t)4 * (((size_t)1 << (2 * level)) - 1) + pix;
    const float4 h = __ldg(&A.dir_tab[2 * idx]);
    const float4 l = __ldg(&A.dir_tab[2 * idx + 1]);
    n[0] = {h.x, l.x};
    n[1] = {h.y, l.y};
    n[2] = {h.z, l.z};
    return h.w != 0.0f;
  }
  double v[3];
  const int diag = pix2vec64(level, pix, v);
  for (int i = 0; i < 3; ++i) {
    const float hi = (float)v[i];
    n[i] = {hi, (float)(v[i] - (double)hi)};
  }
  return diag;
}

// Exact (FP64) crossing decision for cell (c0, c1, c2) of package (level,
// pix) of source src: bit 3 = split, bits 0-2 = axes that reach the next
// plane first, bit 6 = the crossing lies beyond the halting radius rlim
// (+inf without a finite speed of light).  A free function taking values,
// so that calling it does not force the caller's walker state into local
// memory.
__device__ __noinline__ int decide64(const TraceArgs& A, uint32_t src, int level, uint32_t pix, int c0, int c1,
                                     int c2, double rlim) {
  const SourceDev& S = A.src[src];
  double n[3];
  pix2vec64(level, pix, n);
  const double u0 = next_t64(c0, S.s[0], n[0]);
  const double u1 = next_t64(c1, S.s[1], n[1]);
  const double u2 = next_t64(c2, S.s[2], n[2]);
  const double rn = fmin(u0, fmin(u1, u2));
  int out = 0;
  if (level < A.max_level && rn > A.rsplit[level]) out |= 8;
  if (rn > rlim) out |= 64;
  if (n[0] != 0 && u0 == rn) out |= 1;
  if (n[1] != 0 && u1 == rn) out |= 2;
  if (n[2] != 0 && u2 == rn) out |= 4;
  return out;
}

struct Walk32 {
  using Rec = Rec32;  // packages in flight between traces; records of FSL traces
  template <bool FSL> using Q = typename std::conditional<FSL, Rec32, QRec32>::type;  // queue record
  uint32_t src, pix;
  uint32_t age;         // traces since emission (finite speed of light)
  F2 rlim;              // halting radius of this age
  uint32_t level;       // bits 0-3 level, bit 8: 45-degree ray of an exact source,
                        // bit 9: n_HI stored as FP32 pairs
  F2 r;
  float P, tau, tau_lo, Pstart, tau_err;
  F2 iv0, iv1, iv2;     // 1 / n_i (0 for a vanishing component)
  F2 t0, t1, t2;        // distance to the next plane on each axis
  int c0, c1, c2;
  int nx, ny, nz, steps;
  unsigned nseg;
  float nh, nh_lo;      // n_HI of the current cell (pair), loaded one step ahead
  const float* nhi;
  float* K;
  float* G;

  __device__ __forceinline__ int lvl() const { return (int)(level & 15u); }
  __device__ __forceinline__ int cell_index() const { return c0 + nx * (c1 + ny * c2); }
  __device__ __forceinline__ bool diag_exact() const { return (level & 256u) != 0; }
  __device__ __forceinline__ void load_nh(int idx) {
    if (level & 512u) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(nhi) + idx);
      nh = v.x;
      nh_lo = v.y;
    } else {
      nh = __ldg(&nhi[idx]);
      nh_lo = 0.0f;
    }
  }
  // P of a new package of source S (finite speed of light)
  __device__ __forceinline__ double emit(const SourceDev& S) {
    P = __ldg(&S.sabs32.w);
    return (double)P;
  }
  __device__ __forceinline__ int inst(const TraceArgs& A) const { return A.src[src].inst; }
  __device__ __forceinline__ double unit(const TraceArgs& A) const { return A.src[src].unit; }
  __device__ __forceinline__ bool inside() const {
    return c0 >= 0 && c0 < nx && c1 >= 0 && c1 < ny && c2 >= 0 && c2 < nz;
  }
  // distance from the source to the next plane of cell c along an axis
  __device__ __forceinline__ static F2 next_t(int c, float s_hi, float s_lo, F2 iv) {
    if (iv.hi == 0.0f) return {__int_as_float(0x7f800000), 0.0f};
    const float b = (float)(iv.hi > 0.0f ? c + 1 : c);
    const F2 d0 = two_sum(b, -s_hi);
    const F2 d = fast_two_sum(d0.hi, __fsub_rn(d0.lo, s_lo));
    return f2_mul(d, iv);
  }
  // cell of coordinate u along an axis (tie rule: n > 0 floor, n < 0 ceil - 1)
  __device__ __forceinline__ static int cell_of(F2 u, float n) {
    const int f = f2_floor(u);
    if (n < 0.0f && (float)f == u.hi && u.lo == 0.0f) return f - 1;
    return f;
  }
  __device__ __forceinline__ float band(const TraceArgs& A, F2 t, int axis) const {
    const float4 sa = __ldg(&A.src[src].sabs32);
    const float ab = axis == 0 ? sa.x * fabsf(iv0.hi) : (axis == 1 ? sa.y * fabsf(iv1.hi) : sa.z * fabsf(iv2.hi));
    return fmaf(t.hi, kBandT, ab);
  }

  // Geometry of a package at radius r: direction pairs, first cell (the
  // cell index `cell` when given, else the cell holding the point at r),
  // next crossings.  False when that cell is outside the box.
  template <bool GIVEN = false>
  __device__ __forceinline__ bool start_geom(const TraceArgs& A, uint32_t cell = 0) {
    const SourceDev& S = A.src[src];
    const float4 sh = __ldg(&S.s32);
    const float4 sl = __ldg(&S.slo32);
    const InstDev& I = A.inst[S.inst];
    nx = I.nx; ny = I.ny; nz = I.nz;
    F2 n[3];
    const int diag = dir_pair(A, lvl(), pix, n);
    level = (level & (15u | 512u)) | ((diag && sh.w != 0.0f) ? 256u : 0u);
    iv0 = n[0].hi != 0.0f ? f2_recip(n[0]) : F2{0.0f, 0.0f};
    iv1 = n[1].hi != 0.0f ? f2_recip(n[1]) : F2{0.0f, 0.0f};
    iv2 = n[2].hi != 0.0f ? f2_recip(n[2]) : F2{0.0f, 0.0f};
    if (GIVEN) {
      c0 = (int)(cell % (uint32_t)nx);
      c1 = (int)((cell / (uint32_t)nx) % (uint32_t)ny);
      c2 = (int)(cell / ((uint32_t)nx * (uint32_t)ny));
    } else {
      c0 = cell_of(f2_add(F2{sh.x, sl.x}, f2_mul(r, n[0])), n[0].hi);
      c1 = cell_of(f2_add(F2{sh.y, sl.y}, f2_mul(r, n[1])), n[1].hi);
      c2 = cell_of(f2_add(F2{sh.z, sl.z}, f2_mul(r, n[2])), n[2].hi);
      if (!inside()) return false;
    }
    t0 = next_t(c0, sh.x, sl.x, iv0);
    t1 = next_t(c1, sh.y, sl.y, iv1);
    t2 = next_t(c2, sh.z, sl.z, iv2);
    return true;
  }
  __device__ __forceinline__ void bind(const TraceArgs& A) {
    const SourceDev& S = A.src[src];
    const InstDev& I = A.inst[S.inst];
    // the absorber and accumulators of the package's photon type (Sec. 3.2)
    const int t = S.type;
    nhi = (const float*)(t == 0 ? I.nhi : I.nhe[t - 1]);
    K = (float*)(t == 0 ? I.K : I.Khe[t - 1]);
    G = (float*)(t == 0 ? I.G : I.Ghe[t - 1]);
    level = (level & ~512u) | ((I.flags & kInstNhiPair) ? 512u : 0u);
    Pstart = P;
    steps = 0;
  }
  __device__ __forceinline__ bool start(const TraceArgs& A) {
    bind(A);
    if (!start_geom(A)) return false;
    load_nh(cell_index());
    return true;
  }
  // A package continued from the previous trace: the cell it halted in.
  __device__ __forceinline__ void resume(const TraceArgs& A, uint32_t cell) {
    bind(A);
    start_geom<true>(A, cell);
    load_nh(cell_index());
  }
  __device__ __forceinline__ void set_rlim(const TraceArgs& A) {
    if ((int)age < A.n_ages) {
      const float2 v = __ldg(&A.rlim32[age]);
      rlim = F2{v.x, v.y};
    } else {
      set_status(A.ctl, RT_ERR_STATE);
      rlim = F2{0.0f, 0.0f};
    }
  }

  __device__ __forceinline__ void load(const Rec& q) {
    r = {q.r, q.r_lo}; P = q.P; tau = q.tau; tau_lo = q.tau_lo; tau_err = q.tau_err; src = q.src; pix = q.pix;
    level = q.tag & 15u;
    age = q.age;
  }
  // Record of child cpix (level + 1, P/4, same radius, age, optical depth and
  // its error bound); the level sits in the tag's low bits until publication.
  __device__ __forceinline__ Rec make_child(uint32_t cpix) const {
    Rec c;
    c.r = r.hi; c.r_lo = r.lo; c.P = P * 0.25f; c.tau = tau; c.tau_lo = tau_lo; c.tau_err = tau_err;
    c.src = src; c.pix = cpix; c.tag = (uint32_t)(lvl() + 1); c.age = age;
    return c;
  }
  __device__ __forceinline__ static uint32_t cell_of_record(const Rec& q) { return q.cell; }
  // A halted package as the next trace continues it (one trace older).
  __device__ __forceinline__ void store_halted(Rec* q) const {
    reinterpret_cast<float4*>(&q->r)[0] = make_float4(r.hi, r.lo, P, tau);
    reinterpret_cast<uint4*>(&q->tau_lo)[0] =
        make_uint4(__float_as_uint(tau_lo), __float_as_uint(tau_err), src, pix);
    reinterpret_cast<uint4*>(&q->tag)[0] = make_uint4((uint32_t)lvl(), age + 1, (uint32_t)cell_index(), 0u);
  }
  // Publish a record in the global queue: payload first, then the tag with
  // release semantics.  FSL records (48 B) carry the age and the tag
  // ((epoch << 4) | level); the others (32 B) the level beside the source
  // index and the tag ((epoch & 0xffff) << 16 | tau_err as bf16 rounded up).
  template <bool FSL>
  __device__ __forceinline__ static void publish(Q<FSL>* q, const Rec& c, uint32_t epoch) {
    __stcg(reinterpret_cast<float4*>(&q->r), make_float4(c.r, c.r_lo, c.P, c.tau));
    if constexpr (FSL) {
      __stcg(reinterpret_cast<uint4*>(&q->tau_lo),
             make_uint4(__float_as_uint(c.tau_lo), __float_as_uint(c.tau_err), c.src, c.pix));
      __stcg(&q->age, c.age);
      st_release_u32(&q->tag, (epoch << 4) | (c.tag & 15u));
    } else {
      // tau_err >= 0: adding 0xffff before the shift rounds the magnitude up
      const uint32_t e16 = (__float_as_uint(c.tau_err) + 0xffffu) >> 16;
      __stcg(reinterpret_cast<uint2*>(&q->tau_lo), make_uint2(__float_as_uint(c.tau_lo), c.src | ((c.tag & 15u) << 28)));
      __stcg(&q->pix, c.pix);
      st_release_u32(&q->tag, (epoch << 16) | e16);
    }
  }
  // Poll with an acquire load of the tag: the payload reads that follow a
  // successful poll are ordered after it without a fence.
  template <bool FSL>
  __device__ __forceinline__ static bool poll(const Q<FSL>* q, uint32_t epoch, Rec& o) {
    const uint32_t tg = ld_acquire_u32(&q->tag);
    if constexpr (FSL) {
      if ((tg >> 4) != (epoch & 0x0fffffffu)) return false;
    } else {
      if ((tg >> 16) != (epoch & (uint32_t)kEpochMask)) return false;
    }
    const float4 a = __ldcg(reinterpret_cast<const float4*>(&q->r));
    const uint4 b = __ldcg(reinterpret_cast<const uint4*>(&q->tau_lo));
    o.r = a.x; o.r_lo = a.y; o.P = a.z; o.tau = a.w;
    o.tau_lo = __uint_as_float(b.x);
    if constexpr (FSL) {
      o.tau_err = __uint_as_float(b.y); o.src = b.z; o.pix = b.w; o.tag = tg;
      o.age = __ldcg(&q->age);
    } else {
      o.src = b.y & (kMaxQueueSources - 1u); o.tag = b.y >> 28; o.pix = b.z;
      o.tau_err = __uint_as_float(tg << 16);
      o.age = 0u;
    }
    return true;
  }
  // Every lane takes the record that lane `from` holds (all lanes call it).
  __device__ __forceinline__ static void shfl_rec(Rec& c, int from) {
    c.r = __shfl_sync(0xffffffffu, c.r, from);
    c.r_lo = __shfl_sync(0xffffffffu, c.r_lo, from);
    c.P = __shfl_sync(0xffffffffu, c.P, from);
    c.tau = __shfl_sync(0xffffffffu, c.tau, from);
    c.tau_lo = __shfl_sync(0xffffffffu, c.tau_lo, from);
    c.tau_err = __shfl_sync(0xffffffffu, c.tau_err, from);
    c.src = __shfl_sync(0xffffffffu, c.src, from);
    c.pix = __shfl_sync(0xffffffffu, c.pix, from);
    c.tag = __shfl_sync(0xffffffffu, c.tag, from);
    c.age = __shfl_sync(0xffffffffu, c.age, from);
  }
  __device__ __forceinline__ static Rec root_rec(uint32_t gsrc, uint32_t l, uint32_t p) {
    Rec c;
    c.r = 0.0f; c.r_lo = 0.0f; c.P = 1.0f; c.tau = 0.0f; c.tau_lo = 0.0f; c.tau_err = 0.0f; c.src = gsrc; c.pix = p;
    c.tag = l;
    c.age = 0u;
    return c;
  }
  __device__ __forceinline__ void become_child0() {
    level = (uint32_t)(lvl() + 1); pix = 4u * pix; P = P * 0.25f;
  }

  // The next crossing as the FP64 evaluation takes it: bits 0-2 the planes
  // crossed, bit 3 a split first, bits 4-5 the axis of the smallest pair,
  // bit 6 (FSL) the crossing lies beyond the halting radius; rn_out receives
  // the crossing distance.  Orders the pairs cannot prove are re-taken in
  // FP64 (decide64) and counted in fb.
  template <bool FSL>
  __device__ __forceinline__ int decide(const TraceArgs& A, F2& rn_out, unsigned& fb) const {
    // next crossing: the smallest pair, and whether the order is provable
    int imin = 0;
    F2 rn = t0;
    if (f2_less(t1, rn)) { rn = t1; imin = 1; }
    if (f2_less(t2, rn)) { rn = t2; imin = 2; }
    bool m0 = imin == 0, m1 = imin == 1, m2 = imin == 2;
    bool unsure = false;
    const float close = fmaf(rn.hi, kClose, rn.hi) + 1e-30f;
    const bool c_0 = imin != 0 && iv0.hi != 0.0f && t0.hi <= close;
    const bool c_1 = imin != 1 && iv1.hi != 0.0f && t1.hi <= close;
    const bool c_2 = imin != 2 && iv2.hi != 0.0f && t2.hi <= close;
    const int l = lvl();
    const float R = A.rsplit32[l];
    const bool can_split = l < A.max_level;
    const bool split_close = can_split && !(rn.hi > fmaf(R, kClose, R)) && !(rn.hi < fmaf(R, -kClose, R));
    bool split = can_split && rn.hi > R;
    // Step 3j: the crossing against the halting radius, decided like the split
    bool halt = FSL && rn.hi > rlim.hi;
    const bool halt_close = FSL && !(rn.hi > fmaf(rlim.hi, kClose, rlim.hi)) &&
                            !(rn.hi < fmaf(rlim.hi, -kClose, rlim.hi));
    if (c_0 || c_1 || c_2 || split_close || halt_close) {
      // a close pair: compare exactly, re-take the decision in FP64 if unprovable
      const float emin = band(A, rn, imin);
      const bool xy_tie = diag_exact() && f2_eq(t0, t1);
      if (c_0 && f2_diff(t0, rn) <= band(A, t0, 0) + emin) { if (imin == 1 && xy_tie) m0 = true; else unsure = true; }
      if (c_1 && f2_diff(t1, rn) <= band(A, t1, 1) + emin) { if (imin == 0 && xy_tie) m1 = true; else unsure = true; }
      if (c_2 && f2_diff(t2, rn) <= band(A, t2, 2) + emin) unsure = true;
      if (split_close) {
        const float d = f2_diff(rn, F2{R, A.rsplit32lo[l]});
        const float bnd = emin + R * kBandT;
        if (d > bnd) split = true;
        else if (-d > bnd) split = false;
        else unsure = true;
      }
      if (halt_close) {
        const float d = f2_diff(rn, rlim);
        const float bnd = emin + rlim.hi * kBandT;
        if (d > bnd) halt = true;
        else if (-d > bnd) halt = false;
        else unsure = true;
      }
      if (unsure) {
        const double rlim64 = !FSL ? __longlong_as_double(0x7ff0000000000000LL)
                                   : ((int)age < A.n_ages ? A.rlim64[age] : 0.0);
        const int d64 = decide64(A, src, l, pix, c0, c1, c2, rlim64);
        split = (d64 & 8) != 0;
        halt = (d64 & 64) != 0;
        m0 = (d64 & 1) != 0;
        m1 = (d64 & 2) != 0;
        m2 = (d64 & 4) != 0;
        ++fb;
      }
    }
    rn_out = rn;
    return (m0 ? 1 : 0) | (m1 ? 2 : 0) | (m2 ? 4 : 0) | (split ? 8 : 0) | (imin << 4) | (halt ? 64 : 0);
  }
  // Cross the planes of `m` (bits 0-2) at distance rn.
  // The first crossed axis is selected rather than branched on, so the lanes
  // of a warp (crossing different axes) evaluate one next_t together; a
  // second or third axis crossed at the same point (edges, corners) is rare.
  __device__ __forceinline__ void advance(const TraceArgs& A, int m, F2 rn) {
    const int mm = m & 7;
    if (mm) {
      const float4 sh = __ldg(&A.src[src].s32);
      const float4 sl = __ldg(&A.src[src].slo32);
      const int a = (mm & 1) ? 0 : ((mm & 2) ? 1 : 2);
      const F2 iv = a == 0 ? iv0 : (a == 1 ? iv1 : iv2);
      const int c = (a == 0 ? c0 : (a == 1 ? c1 : c2)) + (iv.hi > 0.0f ? 1 : -1);
      const F2 t = next_t(c, a == 0 ? sh.x : (a == 1 ? sh.y : sh.z), a == 0 ? sl.x : (a == 1 ? sl.y : sl.z), iv);
      if (a == 0) { c0 = c; t0 = t; }
      else if (a == 1) { c1 = c; t1 = t; }
      else { c2 = c; t2 = t; }
      const int rest = mm & ~(1 << a);
      if (rest) {
        if (rest & 2) { c1 += iv1.hi > 0.0f ? 1 : -1; t1 = next_t(c1, sh.y, sl.y, iv1); }
        if (rest & 4) { c2 += iv2.hi > 0.0f ? 1 : -1; t2 = next_t(c2, sh.z, sl.z, iv2); }
      }
    }
    r = rn;
  }

  template <bool FSL>
  __device__ __forceinline__ int step(const TraceArgs& A, LaneAcc& acc) {
    F2 rn;
    unsigned fb = 0;
    const int m = decide<FSL>(A, rn, fb);
    acc.fallbacks += fb;
    const int l = lvl();
    if (m & 8) return EV_SPLIT;
    const bool halt = FSL && (m & 64);  // Step 3j: the segment ends at rlim
    // segment length, kappa = sigma dx n_HI and dtau as FP32 pairs: the
    // optical depth (pair) follows the FP64 sum to ~2^-44 where n_HI is a pair
    F2 dr2 = f2_sub(halt ? rlim : rn, r);
    if (dr2.hi < 0.0f) dr2 = F2{0.0f, 0.0f};
    const float dr = dr2.hi;
    const int idx = cell_index();
    const float4 k32 = __ldg(&A.src[src].k32);  // sdx, w, rw, heat
    const F2 kap2 = f2_mul(F2{k32.x, __ldg(&A.src[src].slo32.w)}, F2{nh, nh_lo});
    const F2 dtau2 = f2_mul(kap2, dr2);
    const float kap = kap2.hi;
    const float dtau = dtau2.hi;
    // transmitted fraction tr = e^-tau; phi = (1 - e^-tau)/tau from its Taylor
    // series below tau = 1/4 (7 terms: the first dropped term, tau^7 / 8!, is
    // below 1.6e-9 there, under FP32 rounding), else from tr.
    // Both are computed and one is selected, so lanes do not diverge.
    const float tr = expf(-dtau);
    const float ser = fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(dtau, 1.0f / 5040.0f, -1.0f / 720.0f), dtau, 1.0f / 120.0f), dtau,
                                          -1.0f / 24.0f), dtau, 1.0f / 6.0f), dtau, -0.5f), dtau, 1.0f);
    const float phi = dtau < 0.25f ? ser : __fdividef(1.0f - tr, dtau);
    // covering factor (Eq. "fc"), in FP32 from the pairs' high parts: its
    // error (~1e-4 relative) is far inside the tolerance on k_ph
    float fcv = 1.0f;
    if (A.fc) {
      const float L = r.hi * A.theta32[l];
      if (L > 0.0f) {
        const float4 sh = __ldg(&A.src[src].s32);
        const float rm = fmaf(0.5f, dr, r.hi);
        const float n0 = iv0.hi != 0.0f ? __frcp_rn(iv0.hi) : 0.0f;
        const float n1 = iv1.hi != 0.0f ? __frcp_rn(iv1.hi) : 0.0f;
        const float n2 = iv2.hi != 0.0f ? __frcp_rn(iv2.hi) : 0.0f;
        const float d = fmaxf(fabsf(fmaf(n0, rm, sh.x) - ((float)c0 + 0.5f)),
                              fmaxf(fabsf(fmaf(n1, rm, sh.y) - ((float)c1 + 0.5f)),
                                    fabsf(fmaf(n2, rm, sh.z) - ((float)c2 + 0.5f))));
        const float f = 0.5f + (0.5f - d) / L;
        fcv = fminf(1.0f, f * f);
      }
    }
    const float kadd = P * k32.y * dr * phi * fcv;
    atomicAdd(&K[idx], kadd);
    if (k32.w != 0.0f) atomicAdd(&G[idx], kadd * k32.w);
    if (dr > 0.0f) nseg++;
    P = P * tr;
    {
      const F2 t2 = f2_add(F2{tau, tau_lo}, dtau2);
      tau = t2.hi;
      tau_lo = t2.lo;
    }
    // |tau - tau_FP64| grows by kappa times the pair errors of rn and r (each
    // within 2^-40 rn + 2^-46 |s|/|n| on its axis; twice that, with margin),
    // the rounding of the pair products (2^-37 dtau; 2^-22 dtau where n_HI is
    // plain FP32) and of the pair sum (2^-44 tau)
    {
      const float4 sa = __ldg(&A.src[src].sabs32);
      const float ab = fmaxf(sa.x * fabsf(iv0.hi), fmaxf(sa.y * fabsf(iv1.hi), sa.z * fabsf(iv2.hi)));
      const float e_dtau = (level & 512u) ? 8.0f * kBandT : 4.0f * kEps32;
      tau_err = tau_err + dtau * e_dtau + kap * (fmaf(rn.hi, 4.0f * kBandT, 1e-30f) + 4.0f * ab) +
                tau * (kBandT / 16.0f);
    }
    {
      const float d = f2_diff(F2{tau, tau_lo}, F2{A.tau_term32, A.tau_term32lo});
      const float bnd = tau_err + tau * (4.0f * kBandT) + 1e-30f;
      bool term = d > bnd;
      if (!term && !(-d > bnd)) {
        // too close to call: the lineage's optical depth in FP64 (a lineage
        // emitted in an earlier trace crossed other media, and a cut segment
        // is not the cell's: there the pair's own decision stands)
        const double t64 = (!FSL || (age == 0 && !halt)) ? retrace_tau64(A, src, l, pix, c0, c1, c2)
                                                         : __longlong_as_double(0x7ff8000000000000LL);
        acc.fallbacks_tau++;
        term = isnan(t64) ? (d > 0.0f) : (t64 > A.tau_term);
      }
      if (term) {
        if (nh > 0.0f) {
          const float kres = P * k32.z / nh * fcv;
          atomicAdd(&K[idx], kres);
          if (k32.w != 0.0f) atomicAdd(&G[idx], kres * k32.w);
        }
        acc.absorbed += (double)Pstart * unit(A);
        return EV_DONE;
      }
    }
    if (halt) {
      r = rlim;
      const double u = unit(A);
      acc.absorbed += ((double)Pstart - (double)P) * u;
      acc.halted += (double)P * u;
      return EV_HALT;
    }
    advance(A, m, rn);
    if (!inside()) {
      const double u = unit(A);
      acc.absorbed += ((double)Pstart - (double)P) * u;
      acc.escaped += (double)P * u;
      return EV_DONE;
    }
    // the next cell is known before its density is needed: start the load now
    load_nh(cell_index());
    if (++steps > A.max_steps) {
      set_status(A.ctl, RT_ERR_STATE);
      const double u = unit(A);
      acc.absorbed += ((double)Pstart - (double)P) * u;
      acc.escaped += (double)P * u;
      return EV_DONE;
    }
    return EV_NONE;
  }
  __device__ __forceinline__ void on_split(const TraceArgs& A, LaneAcc& acc) const {
    acc.absorbed += ((double)Pstart - (double)P) * unit(A);
  }
  __device__ __forceinline__ void on_start_outside(const TraceArgs& A, LaneAcc& acc) const {
    acc.escaped += (double)P * unit(A);
  }
};

// ---------------------------------------------------------------------------
// The persistent kernel, generic over the walker.
// ---------------------------------------------------------------------------
template <class W, int MinBlocks, bool FSL>
__global__ void __launch_bounds__(kBlock, MinBlocks) trace_kernel(TraceArgs A) {
  using Rec = typename W::Rec;
  __shared__ unsigned int sh_cnt[kShInst * kLevels];
  __shared__ unsigned long long sh_hsh[kShInst * kLevels];
  __shared__ LaneAcc sh_acc[kBlock];
  __shared__ unsigned int sh_bfb[kShInst * 2];
  for (int i = threadIdx.x; i < kShInst * kLevels; i += blockDim.x) {
    sh_cnt[i] = 0;
    sh_hsh[i] = 0;
  }
  double* const brow = A.blk + (size_t)blockIdx.x * A.blk_rows * kBlkRow;
  for (int i = threadIdx.x; i < A.blk_rows * kBlkRow; i += blockDim.x) brow[i] = 0.0;  // also 0 as an integer
  for (int i = threadIdx.x; i < kShInst * 2; i += blockDim.x) sh_bfb[i] = 0u;
  const BlockBudget BB{brow, A.blk_rows, sh_bfb};
  LaneAcc& acc = sh_acc[threadIdx.x];
  acc.emitted = acc.absorbed = acc.escaped = acc.resumed = acc.halted = 0.0;
  acc.segments = acc.fallbacks = acc.fallbacks_tau = 0;
  acc.inst = -1;
  __syncthreads();
  LevelCounters LC{sh_cnt, sh_hsh};

  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const uint32_t epoch = (uint32_t)A.ctl[CTL_EPOCH];
  using QR = typename W::template Q<FSL>;
  QR* queue = (QR*)A.queue;
  // tickets: roots [0, n_roots), packages in flight [n_roots, qbase), queue slots after
  unsigned long long res_a = 0, n_res = 0;
  if (FSL) {
    res_a = A.ctl[CTL_RES_A];
    n_res = A.ctl[CTL_RES_B] - res_a;
  }
  const unsigned long long qbase = A.n_roots + n_res;

  W w;
  w.nseg = 0;
  bool active = false;
  long long ticket = -1;
  long long seen_out = -1;
  uint64_t seen_ns = global_ns();
  unsigned backoff = 256;  // ns; idle warps back off exponentially up to 4 us

  for (;;) {
    // (1) idle lanes without a ticket take one (one atomic per warp)
    const bool want = !active && ticket < 0;
    const unsigned wm = __ballot_sync(kFull, want);
    if (wm) {
      const int leader = __ffs(wm) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(&A.ctl[CTL_HEAD], (unsigned long long)__popc(wm));
      base = __shfl_sync(kFull, base, leader);
      if (want) ticket = (long long)(base + __popc(wm & lt_mask));
    }
    // (2) turn tickets into packages
    int ev = EV_NONE;
    if (!active && ticket >= 0) {
      const unsigned long long tk = (unsigned long long)ticket;
      bool got = false, resumed = false;
      uint32_t cell = 0;
      if (tk < A.n_roots) {
        const uint32_t ls = (uint32_t)(tk / A.npix0);
        const uint32_t p = (uint32_t)(tk - (unsigned long long)ls * A.npix0);
        const uint32_t gsrc = (uint32_t)A.src_first + ls;
        w.load(W::root_rec(gsrc, (uint32_t)A.level0, p));
        got = true;
        const SourceDev& S = A.src[gsrc];
        acc_switch(acc, w.nseg, S.inst, A, BB);
        if (FSL) acc.emitted += w.emit(S) * S.unit;
        else acc.emitted += S.unit;
        LC.add(A, S.inst, S.local, A.level0, p, 1);
      } else if (FSL && tk < qbase) {
        // a package halted by the previous trace continues from its cell
        const Rec* in = (const Rec*)A.res_in + (res_a + (tk - A.n_roots));
        const Rec q = *in;
        w.load(q);
        cell = W::cell_of_record(q);
        got = resumed = true;
      } else {
        const unsigned long long slot = tk - qbase;
        if (slot < A.cap) {
          Rec q;
          if (W::template poll<FSL>(&queue[slot], epoch, q)) {
            w.load(q);
            got = true;
          }
        }
      }
      if (got) {
        ticket = -1;
        active = true;
        acc_switch(acc, w.nseg, w.inst(A), A, BB);
        if (FSL) w.set_rlim(A);
        if (FSL && resumed) {
          acc.resumed += (double)w.P * w.unit(A);
          w.resume(A, cell);
        } else if (!w.start(A)) {
          w.on_start_outside(A, acc);
          ev = EV_DONE;
        }
      }
    }
    // (3) a warp with nothing to trace checks for the end of the trace
    const unsigned am = __ballot_sync(kFull, active && ev == EV_NONE);
    if (am == 0 && __ballot_sync(kFull, ev == EV_DONE) == 0) {
      long long outst = 0;
      if (lane == 0) outst = (long long)ld_relaxed_u64(&A.ctl[CTL_OUTSTANDING]);
      outst = __shfl_sync(kFull, outst, 0);
      if (outst <= 0) break;
      const uint64_t now = global_ns();
      if (outst != seen_out) {
        seen_out = outst;
        seen_ns = now;
      } else if ((long long)(now - seen_ns) > A.timeout_ns) {
        if (lane == 0) set_status(A.ctl, RT_ERR_TIMEOUT);
        break;
      }
      __nanosleep(backoff);
      backoff = backoff < 4096 ? 2 * backoff : 4096;
      continue;
    }
    backoff = 256;
    seen_out = -1;  // the no-progress clock runs over one idle stretch only
    // (4) trace a few segments
    if (active && ev == EV_NONE) {
      for (int it = 0; it < A.segs_per_iter; ++it) {
        ev = w.template step<FSL>(A, acc);
        if (ev != EV_NONE) break;
      }
    }
    // The lanes left the loop at different steps: reconverge them here, before
    // the warp-wide steps below.  (Without this barrier the same kernel ran
    // 7-11 % slower on every workload measured.)
    __syncwarp();
    // (4b) halted packages go to the output store (one atomic per warp);
    //      from here on they are finished packages
    if (FSL) {
      const unsigned hm = __ballot_sync(kFull, ev == EV_HALT);
      if (hm) {
        const int leader = __ffs(hm) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(&A.ctl[CTL_HALTED], (unsigned long long)__popc(hm));
        base = __shfl_sync(kFull, base, leader);
        if (ev == EV_HALT) {
          const unsigned long long slot = base + __popc(hm & lt_mask);
          if (slot < A.halt_cap) w.store_halted((Rec*)A.halt_out + slot);
          else set_status(A.ctl, RT_ERR_QUEUE_OVERFLOW);
          ev = EV_DONE;
        }
      }
    }
    // (5) a split keeps child 0 and hands children 1-3 first to lanes of this
    //     warp that are free (no package and no ticket: in practice the
    //     lanes whose package ended in this round; a lane holding a ticket
    //     must stay free to take up the record that the ticket names), the
    //     rest to the queue (slots reserved together); finished packages
    //     leave the outstanding count.
    //     One atomic per warp carries both: +3 per split, -1 per finished
    //     package.  Child j = 3 i + k - 1 of the i-th splitting lane goes to
    //     the j-th free lane when there is one, else to slot base + j - nin.
    const bool split = (ev == EV_SPLIT);
    const unsigned sm = __ballot_sync(kFull, split);
    const unsigned dm = __ballot_sync(kFull, ev == EV_DONE);
    if (sm | dm) {
      const int leader = __ffs(sm | dm) - 1;
      const unsigned nsp = __popc(sm);
      // (not in the finite-speed-of-light kernel, which spills at the
      // register cap already: there the hand-off code cost more than it saved)
      const unsigned fm = FSL ? 0u : __ballot_sync(kFull, !split && (!active || ev == EV_DONE) && ticket < 0);
      const unsigned nfree = __popc(fm);
      const unsigned nin = nfree < 3u * nsp ? nfree : 3u * nsp;  // children placed in this warp
      const unsigned nq = 3u * nsp - nin;                         // children through the queue
      unsigned long long base = 0;
      if (lane == leader) {
        // The count must include the children before any child is published,
        // or a consumer could finish a child and see it reach zero: wait for
        // the atomic's return value, then fence.
        const long long delta = 3LL * nsp - (long long)__popc(dm);
        const unsigned long long o = atomicAdd(&A.ctl[CTL_OUTSTANDING], (unsigned long long)delta);
        asm volatile("" ::"l"(o) : "memory");
        if (nq) {
          base = atomicAdd(&A.ctl[CTL_TAIL], (unsigned long long)nq);
          __threadfence();
        }
      }
      base = __shfl_sync(kFull, base, leader);
      if (ev == EV_DONE) {
        active = false;
        ev = EV_NONE;
      }
      bool fresh = false;  // a package starts in this lane now
      if (!FSL && nin) {
        const unsigned q = __popc(fm & lt_mask);
        const bool recv = ((fm >> lane) & 1u) && q < nin;
        Rec c = w.make_child(4u * w.pix);  // in splitting lanes: child 0's record, children differ in pix
        W::shfl_rec(c, recv ? nth_set_bit(sm, q / 3u) : lane);
        if (recv) {
          c.pix += q % 3u + 1u;
          w.load(c);
          active = true;
          fresh = true;
          acc_switch(acc, w.nseg, w.inst(A), A, BB);
          if (FSL) w.set_rlim(A);
        }
      }
      if (split) {
        w.on_split(A, acc);
        const unsigned i = __popc(sm & lt_mask);
        const SourceDev& S = A.src[w.src];
        const int cl = w.lvl() + 1;
        LC.add(A, S.inst, S.local, cl, 4u * w.pix, 4);
        unsigned dropped = 0;
        for (uint32_t k = 1; k < 4; ++k) {
          const unsigned j = 3u * i + (k - 1u);
          if (j < nin) continue;  // placed in a free lane of this warp
          const unsigned long long slot = base + (j - nin);
          if (slot < A.cap) W::template publish<FSL>(&queue[slot], w.make_child(4u * w.pix + k), epoch);
          else ++dropped;
        }
        if (dropped) {
          set_status(A.ctl, RT_ERR_QUEUE_OVERFLOW);
          atomicAdd(&A.ctl[CTL_OUTSTANDING], (unsigned long long)(-(long long)dropped));
        }
        w.become_child0();
        fresh = true;
      }
      if (fresh) {
        if (w.start(A)) ev = EV_NONE;
        else {
          w.on_start_outside(A, acc);
          ev = EV_DONE;
        }
      }
    }
    // (6) a child 0 that starts outside the box is finished too
    const bool done = (ev == EV_DONE);
    const unsigned dm2 = __ballot_sync(kFull, done);
    if (dm2) {
      if (lane == __ffs(dm2) - 1)
        atomicAdd(&A.ctl[CTL_OUTSTANDING], (unsigned long long)(-(long long)__popc(dm2)));
      if (done) active = false;
    }
  }
  acc.segments += w.nseg;
  // Where every lane of the block last worked on the same grid (or on none),
  // reduce the lanes' sums in shared memory first: 256 atomics onto one
  // word would serialise.
  __shared__ int sh_inst;
  if (threadIdx.x == 0) sh_inst = -1;
  __syncthreads();
  if (acc.inst >= 0) atomicMax(&sh_inst, acc.inst);
  __syncthreads();
  if (__syncthreads_and(acc.inst < 0 || acc.inst == sh_inst)) {
    for (int h = kBlock / 2; h > 0; h >>= 1) {
      if (threadIdx.x < h) {
        const LaneAcc& o = sh_acc[threadIdx.x + h];
        acc.emitted += o.emitted;
        acc.absorbed += o.absorbed;
        acc.escaped += o.escaped;
        acc.resumed += o.resumed;
        acc.halted += o.halted;
        acc.segments += o.segments;
        acc.fallbacks += o.fallbacks;
        acc.fallbacks_tau += o.fallbacks_tau;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      acc.inst = sh_inst;
      acc_flush(acc, A, BB);
    }
  } else {
    acc_flush(acc, A, BB);
  }
  // the block's reductions into its rows are complete and visible before
  // the rows are read back (from L2)
  __threadfence();
  __syncthreads();
  for (int i = threadIdx.x; i < A.blk_rows; i += blockDim.x) {
    const InstDev& I = A.inst[i];
    for (int k = 0; k < kAcc; ++k) {
      const double v = __ldcg(&brow[kBlkRow * i + k]);
      if (v != 0.0) atomicAdd(&I.acc[k], v);
    }
    const unsigned long long sg = __ldcg(reinterpret_cast<const unsigned long long*>(&brow[kBlkRow * i + kAcc]));
    if (sg) atomicAdd(&I.cnt[kCntSegments], sg);
    if (sh_bfb[2 * i]) atomicAdd(&I.cnt[kCntFallbacks], (unsigned long long)sh_bfb[2 * i]);
    if (sh_bfb[2 * i + 1]) atomicAdd(&I.cnt[kCntFallbacksTau], (unsigned long long)sh_bfb[2 * i + 1]);
  }
  for (int i = threadIdx.x; i < kShInst * kLevels; i += blockDim.x) {
    const int inst = i / kLevels, l = i - inst * kLevels;
    if (inst < A.ninst && sh_cnt[i]) {
      atomicAdd(&A.inst[inst].cnt[l], (unsigned long long)sh_cnt[i]);
      atomicAdd(&A.inst[inst].cnt[kLevels + l], sh_hsh[i]);
    }
  }
}

constexpr int kInitBlocks = 16;  // blocks of trace_init_kernel (they clear the queue at an epoch wrap)

// Resets the queue for pass `pass` of `passes`.  A trace may run as several
// passes over ranges of its sources; the status of earlier passes stays (the
// first error wins) and their queue use is folded into CTL_PEAK / CTL_PUSHED.
// Packages in flight (finite speed of light): at the first pass, mode
// FLIGHT_ADVANCE takes what the previous trace halted (at most in_cap
// records were stored) as this trace's input; every pass continues an equal
// share of them.
//
// Every pass takes the next epoch, and queue records carry its low 16 bits
// (QRec32).  Before an epoch whose low 16 bits would be 0 the launch clears
// the queue (all blocks, grid-stride) and takes the epoch after it: a record
// left in a slot that no trace has written for 2^16 - 1 epochs cannot then
// pass for a current one, and zeroed memory never does.  Every block reads
// the old epoch before it counts itself done in CTL_INIT_DONE; the block that
// counts last writes the control words (no block waits on another).
__global__ void trace_init_kernel(unsigned long long* ctl, uint4* queue, unsigned long long queue_u4,
                                  unsigned long long n_roots, int first_pass, int mode, unsigned long long in_cap,
                                  int pass, int passes) {
  __shared__ unsigned long long s_epoch;
  __shared__ int s_last;
  if (threadIdx.x == 0) s_epoch = *(volatile unsigned long long*)&ctl[CTL_EPOCH];
  __syncthreads();
  const unsigned long long old = s_epoch;
  const bool wrap = ((old + 1) & kEpochMask) == 0;
  if (wrap && queue) {
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < queue_u4;
         i += (unsigned long long)gridDim.x * blockDim.x)
      queue[i] = z;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&ctl[CTL_INIT_DONE], 1ULL) == (unsigned long long)gridDim.x - 1ULL;
  }
  __syncthreads();
  if (threadIdx.x != 0 || !s_last) return;
  __threadfence();
  ctl[CTL_INIT_DONE] = 0;
  if (first_pass) {
    // a state rejected by an asynchronous upload stays reported until the
    // host has read it
    ctl[CTL_STATUS] = ctl[CTL_SET_ERR];
    ctl[CTL_PEAK] = 0;
    ctl[CTL_PUSHED] = 0;
    if (mode == FLIGHT_OFF) ctl[CTL_RESUME] = 0;
    else if (mode == FLIGHT_ADVANCE) ctl[CTL_RESUME] = ctl[CTL_HALTED] < in_cap ? ctl[CTL_HALTED] : in_cap;
    ctl[CTL_HALTED] = 0;
  } else {
    const unsigned long long t = ctl[CTL_TAIL];
    if (t > ctl[CTL_PEAK]) ctl[CTL_PEAK] = t;
    ctl[CTL_PUSHED] += t;
  }
  const unsigned long long nr = ctl[CTL_RESUME];
  const unsigned long long a = nr * (unsigned long long)pass / (unsigned long long)passes;
  const unsigned long long b = nr * (unsigned long long)(pass + 1) / (unsigned long long)passes;
  ctl[CTL_RES_A] = a;
  ctl[CTL_RES_B] = b;
  ctl[CTL_HEAD] = 0;
  ctl[CTL_TAIL] = 0;
  ctl[CTL_OUTSTANDING] = n_roots + (b - a);
  ctl[CTL_EPOCH] = old + (wrap ? 2ULL : 1ULL);
}

// Host-side launch helpers (called from api.cu).  `queue` / `queue_bytes`:
// the whole queue allocation (a multiple of 16 bytes), cleared when the epoch
// wraps.
cudaError_t launch_trace_init(unsigned long long* ctl, void* queue, size_t queue_bytes, unsigned long long n_roots,
                              int first_pass, int mode, unsigned long long in_cap, int pass, int passes,
                              cudaStream_t st) {
  if (queue_bytes % 16 != 0 || ((uintptr_t)queue & 15u) != 0) return cudaErrorInvalidValue;
  trace_init_kernel<<<kInitBlocks, 256, 0, st>>>(ctl, (uint4*)queue, queue_bytes / 16, n_roots, first_pass, mode,
                                                in_cap, pass, passes);
  return cudaGetLastError();
}

// Halting radii of the next trace from those of the previous one (finite
// speed of light): neu[0] = c_dt, neu[a] = old[a - 1] + c_dt, FP64, and
// their FP32 pairs.
__global__ void flight_table_kernel(const double* old, double* neu, float2* neu32, int n_new, double c_dt) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n_new; a += gridDim.x * blockDim.x) {
    const double v = a == 0 ? c_dt : __dadd_rn(old[a - 1], c_dt);
    neu[a] = v;
    const float hi = __double2float_rn(v);
    neu32[a] = make_float2(hi, __double2float_rn(__dsub_rn(v, (double)hi)));
  }
}

cudaError_t launch_flight_table(const double* old, double* neu, float2* neu32, int n_new, double c_dt,
                                cudaStream_t st) {
  flight_table_kernel<<<(n_new + 255) / 256, 256, 0, st>>>(old, neu, neu32, n_new, c_dt);
  return cudaGetLastError();
}

constexpr int kMinBlocks64 = 2;
constexpr int kMinBlocks32 = TRACE_MIN_BLOCKS;

cudaError_t trace_occupancy(int precision, int fsl, int block, int* blocks_per_sm) {
  if (block != kBlock) return cudaErrorInvalidValue;
  if (precision == RT_FP64)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm,
        fsl ? trace_kernel<Walk64, kMinBlocks64, true> : trace_kernel<Walk64, kMinBlocks64, false>, block, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      blocks_per_sm, fsl ? trace_kernel<Walk32, kMinBlocks32, true> : trace_kernel<Walk32, kMinBlocks32, false>,
      block, 0);
}

// fsl: the finite-speed-of-light instantiation (A.rlim*, res_in, halt_out set)
cudaError_t launch_trace(int precision, int fsl, const TraceArgs& A, int grid, int block, cudaStream_t st) {
  if (block != kBlock) return cudaErrorInvalidValue;
  if (precision == RT_FP64) {
    if (fsl) trace_kernel<Walk64, kMinBlocks64, true><<<grid, block, 0, st>>>(A);
    else trace_kernel<Walk64, kMinBlocks64, false><<<grid, block, 0, st>>>(A);
  } else {
    if (fsl) trace_kernel<Walk32, kMinBlocks32, true><<<grid, block, 0, st>>>(A);
    else trace_kernel<Walk32, kMinBlocks32, false><<<grid, block, 0, st>>>(A);
  }
  return cudaGetLastError();
}

// Direction table: for each pixel of levels 0..L (level l starts at entry
// 4 (4^l - 1)), two float4: (hi.x, hi.y, hi.z, diag) and (lo.x, lo.y, lo.z, 0)
// with hi + lo the FP64 direction of pix2vec64.
__global__ void direction_table_kernel(int level, float4* tab) {
  const unsigned long long npix = 12ULL << (2 * level);
  const size_t base = (size_t)4 * (((size_t)1 << (2 * level)) - 1);
  for (unsigned long long p = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; p < npix;
       p += (unsigned long long)gridDim.x * blockDim.x) {
    double v[3];
    const int diag = pix2vec64(level, (uint32_t)p, v);
    float hi[3], lo[3];
    for (int i = 0; i < 3; ++i) {
      hi[i] = (float)v[i];
      lo[i] = (float)(v[i] - (double)hi[i]);
    }
    tab[2 * (base + p)] = make_float4(hi[0], hi[1], hi[2], diag ? 1.0f : 0.0f);
    tab[2 * (base + p) + 1] = make_float4(lo[0], lo[1], lo[2], 0.0f);
  }
}

cudaError_t launch_direction_table(int level, float4* tab, cudaStream_t st) {
  direction_table_kernel<<<152 * 8, 256, 0, st>>>(level, tab);
  return cudaGetLastError();
}

// Self-check of the FP32 direction bound: max over the pixels of `level` of
// max_i |n32_i - n64_i|, written to out[0] (as the bit pattern of a positive
// double, so atomicMax on the integer view orders it correctly).
__global__ void direction_error_kernel(int level, unsigned long long* out) {
  const unsigned long long npix = 12ULL << (2 * level);
  double worst = 0.0;
  for (unsigned long long p = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; p < npix;
       p += (unsigned long long)gridDim.x * blockDim.x) {
    double n64[3];
    float n32[3];
    pix2vec64(level, (uint32_t)p, n64);
    pix2vec32(level, (uint32_t)p, n32);
    for (int i = 0; i < 3; ++i) worst = fmax(worst, fabs((double)n32[i] - n64[i]));
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(worst));
}

cudaError_t launch_direction_check(int level, unsigned long long* out, cudaStream_t st) {
  direction_error_kernel<<<152 * 8, 256, 0, st>>>(level, out);
  return cudaGetLastError();
}

}  // namespace rtg
