// trace.cu -- persistent ray-tracing kernel (Sec. 2.1-2.2, Steps 1-5 of
// Sec. 3.1) for one or many grids at once.
//
// Work model.  Every lane of the persistent grid carries at most one photon
// package.  A lane without a package takes a ticket from a global counter
// (one atomic per warp).  Tickets below n_roots are root packages (Step 1:
// source = ticket / N_pix, pixel = ticket % N_pix, P = 1 in units of the
// source's Ndot / N_pix) and need no memory; higher tickets name queue slots
// that split packages publish.  When a package splits (Step 3e) its lane
// keeps child 0 and appends children 1-3 to the queue (one atomic per warp
// reserves the slots); each record's tag word is stored last with release
// semantics and read with acquire semantics.  An outstanding-package counter
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
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "healpix.cuh"
#include "rt_internal.cuh"

namespace rtg {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kShInst = 16;  // grids whose level counters are kept in shared memory

enum Event { EV_NONE = 0, EV_SPLIT = 1, EV_DONE = 2 };

struct LaneAcc {
  int inst;
  double emitted, absorbed, escaped;
  unsigned int segments;
  unsigned int fallbacks;
};

__device__ __forceinline__ void acc_flush(LaneAcc& a, const TraceArgs& A) {
  if (a.inst >= 0) {
    const InstDev& I = A.inst[a.inst];
    if (a.emitted != 0.0) atomicAdd(&I.acc[0], a.emitted);
    if (a.absorbed != 0.0) atomicAdd(&I.acc[1], a.absorbed);
    if (a.escaped != 0.0) atomicAdd(&I.acc[2], a.escaped);
    if (a.segments) atomicAdd(&I.cnt[kCntSegments], (unsigned long long)a.segments);
    if (a.fallbacks) atomicAdd(&I.cnt[kCntFallbacks], (unsigned long long)a.fallbacks);
  }
  a.emitted = a.absorbed = a.escaped = 0.0;
  a.segments = 0;
  a.fallbacks = 0;
}

__device__ __forceinline__ void acc_switch(LaneAcc& a, int inst, const TraceArgs& A) {
  if (a.inst != inst) {
    acc_flush(a, A);
    a.inst = inst;
  }
}

struct LevelCounters {
  unsigned int* cnt;        // [kShInst][kLevels]
  unsigned long long* hsh;  // [kShInst][kLevels]
  __device__ __forceinline__ void add(const TraceArgs& A, int inst, int local, int level, uint32_t pix) {
    const unsigned long long h = pkg_hash((uint32_t)local, (uint32_t)level, pix);
    if (inst < kShInst) {
      atomicAdd(&cnt[inst * kLevels + level], 1u);
      atomicAdd(&hsh[inst * kLevels + level], h);
    } else {
      atomicAdd(&A.inst[inst].cnt[level], 1ULL);
      atomicAdd(&A.inst[inst].cnt[kLevels + level], h);
    }
  }
};

// ---------------------------------------------------------------------------
// FP64 walker: every decision (cell of a point, next crossing, split,
// termination) is evaluated with explicitly rounded FP64 operations in the
// order a plain FP64 evaluation of the method's formulas uses.
// ---------------------------------------------------------------------------
struct Walk64 {
  using Rec = Rec64;
  uint32_t src, level, pix;
  int inst, local;
  double r, P, tau, Pstart;
  double s0, s1, s2, n0, n1, n2, t0, t1, t2;
  int c0, c1, c2;
  int nx, ny, nz, steps;
  const double* nhi;
  double* K;
  double* G;
  double sdx, w, rw, heat, unit;

  __device__ __forceinline__ static int cell_of(double u, double n) {
    if (n > 0) return (int)floor(u);
    if (n < 0) return (int)ceil(u) - 1;
    return (int)floor(u);
  }
  __device__ __forceinline__ static double next_t(int c, double s, double n) {
    if (n > 0) return __ddiv_rn(__dsub_rn((double)(c + 1), s), n);
    if (n < 0) return __ddiv_rn(__dsub_rn((double)c, s), n);
    return __longlong_as_double(0x7ff0000000000000LL);  // +inf
  }
  __device__ __forceinline__ bool inside() const {
    return c0 >= 0 && c0 < nx && c1 >= 0 && c1 < ny && c2 >= 0 && c2 < nz;
  }

  // Steps 3a-3b: direction and cell at radius r.  Returns false if the
  // package starts outside the box.
  __device__ __forceinline__ bool start(const TraceArgs& A) {
    const SourceDev& S = A.src[src];
    inst = S.inst;
    local = S.local;
    s0 = S.s[0]; s1 = S.s[1]; s2 = S.s[2];
    sdx = S.sdx; w = S.w; rw = S.rw; heat = S.heat; unit = S.unit;
    const InstDev& I = A.inst[inst];
    nx = I.nx; ny = I.ny; nz = I.nz;
    nhi = (const double*)I.nhi;
    K = (double*)I.K;
    G = (double*)I.G;
    double n[3];
    pix2vec64((int)level, pix, n);
    n0 = n[0]; n1 = n[1]; n2 = n[2];
    c0 = cell_of(__dadd_rn(s0, __dmul_rn(r, n0)), n0);
    c1 = cell_of(__dadd_rn(s1, __dmul_rn(r, n1)), n1);
    c2 = cell_of(__dadd_rn(s2, __dmul_rn(r, n2)), n2);
    Pstart = P;
    steps = 0;
    if (!inside()) return false;
    t0 = next_t(c0, s0, n0);
    t1 = next_t(c1, s1, n1);
    t2 = next_t(c2, s2, n2);
    return true;
  }

  __device__ __forceinline__ void load(const Rec& q) {
    r = q.r; P = q.P; tau = q.tau; src = q.src; pix = q.pix; level = q.level;
  }
  __device__ __forceinline__ void store_child(Rec* q, uint32_t cpix, uint32_t epoch) const {
    __stcg(&q->r, r);
    __stcg(&q->P, P * 0.25);
    __stcg(&q->tau, tau);
    __stcg(&q->src, src);
    __stcg(&q->pix, cpix);
    __stcg(&q->level, level + 1);
    st_release_u32(&q->tag, epoch);
  }
  __device__ __forceinline__ static void read_rec(const Rec* q, Rec& o) {
    o.r = __ldcg(&q->r); o.P = __ldcg(&q->P); o.tau = __ldcg(&q->tau);
    o.src = __ldcg(&q->src); o.pix = __ldcg(&q->pix); o.level = __ldcg(&q->level);
  }
  __device__ __forceinline__ void set_root(uint32_t gsrc, uint32_t lvl, uint32_t p) {
    src = gsrc; level = lvl; pix = p; r = 0.0; P = 1.0; tau = 0.0;
  }
  __device__ __forceinline__ void become_child0() {
    level += 1; pix = 4u * pix; P = P * 0.25;
  }
  __device__ __forceinline__ double p_physical(double p) const { return p * unit; }

  // One segment.  Returns EV_SPLIT before traversing a cell whose exit radius
  // exceeds R_split, EV_DONE when the package is absorbed or leaves the box.
  __device__ __forceinline__ int step(const TraceArgs& A, LaneAcc& acc) {
    const double rn = fmin(t0, fmin(t1, t2));
    if ((int)level < A.max_level && rn > A.rsplit[level]) return EV_SPLIT;
    double dr = __dsub_rn(rn, r);
    if (dr < 0) dr = 0;
    const int idx = c0 + nx * (c1 + ny * c2);
    const double nh = __ldg(&nhi[idx]);
    const double dtau = __dmul_rn(__dmul_rn(sdx, nh), dr);
    const double am = -expm1(-dtau);
    const double phi = dtau > 0 ? am / dtau : 1.0;
    const double kadd = P * w * dr * phi;
    atomicAdd(&K[idx], kadd);
    if (heat != 0.0) atomicAdd(&G[idx], kadd * heat);
    if (dr > 0) acc.segments++;
    P = P - P * am;
    tau = __dadd_rn(tau, dtau);
    if (tau > A.tau_term) {
      const double kres = P * rw / nh;
      atomicAdd(&K[idx], kres);
      if (heat != 0.0) atomicAdd(&G[idx], kres * heat);
      acc.absorbed += Pstart * unit;
      return EV_DONE;
    }
    if (n0 != 0 && t0 == rn) { c0 += n0 > 0 ? 1 : -1; t0 = next_t(c0, s0, n0); }
    if (n1 != 0 && t1 == rn) { c1 += n1 > 0 ? 1 : -1; t1 = next_t(c1, s1, n1); }
    if (n2 != 0 && t2 == rn) { c2 += n2 > 0 ? 1 : -1; t2 = next_t(c2, s2, n2); }
    r = rn;
    if (!inside()) {
      acc.absorbed += (Pstart - P) * unit;
      acc.escaped += P * unit;
      return EV_DONE;
    }
    if (++steps > A.max_steps) {
      set_status(A.ctl, RT_ERR_STATE);
      acc.absorbed += (Pstart - P) * unit;
      acc.escaped += P * unit;
      return EV_DONE;
    }
    return EV_NONE;
  }
  // Budget of the parent's run when it splits (children carry P/4 each).
  __device__ __forceinline__ void on_split(LaneAcc& acc) const { acc.absorbed += (Pstart - P) * unit; }
  __device__ __forceinline__ void on_start_outside(LaneAcc& acc) const { acc.escaped += P * unit; }
};

// ---------------------------------------------------------------------------
// The persistent kernel, generic over the walker.
// ---------------------------------------------------------------------------
template <class W>
__global__ void __launch_bounds__(256) trace_kernel(TraceArgs A) {
  using Rec = typename W::Rec;
  __shared__ unsigned int sh_cnt[kShInst * kLevels];
  __shared__ unsigned long long sh_hsh[kShInst * kLevels];
  for (int i = threadIdx.x; i < kShInst * kLevels; i += blockDim.x) {
    sh_cnt[i] = 0;
    sh_hsh[i] = 0;
  }
  __syncthreads();
  LevelCounters LC{sh_cnt, sh_hsh};

  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const uint32_t epoch = (uint32_t)A.ctl[CTL_EPOCH];
  Rec* queue = (Rec*)A.queue;

  W w;
  bool active = false;
  long long ticket = -1;
  LaneAcc acc{-1, 0.0, 0.0, 0.0, 0u, 0u};
  long long seen_out = -1;
  uint64_t seen_ns = global_ns();

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
      bool got = false;
      if (tk < A.n_roots) {
        const uint32_t gsrc = (uint32_t)(tk / A.npix0);
        const uint32_t p = (uint32_t)(tk - (unsigned long long)gsrc * A.npix0);
        w.set_root(gsrc, (uint32_t)A.level0, p);
        got = true;
        const SourceDev& S = A.src[gsrc];
        acc_switch(acc, S.inst, A);
        acc.emitted += S.unit;
        LC.add(A, S.inst, S.local, A.level0, p);
      } else {
        const unsigned long long slot = tk - A.n_roots;
        if (slot < A.cap && ld_acquire_u32(&queue[slot].tag) == epoch) {
          Rec q;
          W::read_rec(&queue[slot], q);
          w.load(q);
          got = true;
        }
      }
      if (got) {
        ticket = -1;
        active = true;
        if (!w.start(A)) {
          acc_switch(acc, w.inst, A);
          w.on_start_outside(acc);
          ev = EV_DONE;
        } else {
          acc_switch(acc, w.inst, A);
        }
      }
    }
    // (3) a warp with nothing to trace checks for the end of the trace
    const unsigned am = __ballot_sync(kFull, active && ev == EV_NONE);
    if (am == 0 && __ballot_sync(kFull, ev == EV_DONE) == 0) {
      long long outst = 0;
      if (lane == 0) outst = ld_acquire_s64(&A.ctl[CTL_OUTSTANDING]);
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
      __nanosleep(128);
      continue;
    }
    // (4) trace a few segments
    if (active && ev == EV_NONE) {
      for (int it = 0; it < A.segs_per_iter; ++it) {
        ev = w.step(A, acc);
        if (ev != EV_NONE) break;
      }
    }
    // (5) splits: reserve 3 slots per splitting lane, publish children 1-3,
    //     keep child 0
    const bool split = (ev == EV_SPLIT);
    const unsigned sm = __ballot_sync(kFull, split);
    if (sm) {
      const int leader = __ffs(sm) - 1;
      const unsigned nsp = __popc(sm);
      unsigned long long base = 0;
      if (lane == leader) {
        // The increment must be performed before any child is published, or
        // a consumer could finish a child and see the count reach zero: wait
        // for the atomic's return value, then fence.
        const unsigned long long o = atomicAdd(&A.ctl[CTL_OUTSTANDING], 3ULL * nsp);
        asm volatile("" ::"l"(o) : "memory");
        base = atomicAdd(&A.ctl[CTL_TAIL], 3ULL * nsp);
        __threadfence();
      }
      base = __shfl_sync(kFull, base, leader);
      if (split) {
        w.on_split(acc);
        const unsigned long long my = base + 3ULL * __popc(sm & lt_mask);
        const uint32_t cl = w.level + 1;
        for (uint32_t k = 0; k < 4; ++k) LC.add(A, w.inst, w.local, (int)cl, 4u * w.pix + k);
        unsigned dropped = 0;
        for (uint32_t k = 1; k < 4; ++k) {
          const unsigned long long slot = my + (k - 1);
          if (slot < A.cap) w.store_child(&queue[slot], 4u * w.pix + k, epoch);
          else ++dropped;
        }
        if (dropped) {
          set_status(A.ctl, RT_ERR_QUEUE_OVERFLOW);
          atomicAdd(&A.ctl[CTL_OUTSTANDING], (unsigned long long)(-(long long)dropped));
        }
        w.become_child0();
        if (w.start(A)) ev = EV_NONE;
        else {
          w.on_start_outside(acc);
          ev = EV_DONE;
        }
      }
    }
    // (6) finished packages leave the outstanding count
    const bool done = (ev == EV_DONE);
    const unsigned dm = __ballot_sync(kFull, done);
    if (dm) {
      if (lane == __ffs(dm) - 1)
        atomicAdd(&A.ctl[CTL_OUTSTANDING], (unsigned long long)(-(long long)__popc(dm)));
      if (done) active = false;
    }
  }
  acc_flush(acc, A);
  __syncthreads();
  for (int i = threadIdx.x; i < kShInst * kLevels; i += blockDim.x) {
    const int inst = i / kLevels, l = i - inst * kLevels;
    if (inst < A.ninst && sh_cnt[i]) {
      atomicAdd(&A.inst[inst].cnt[l], (unsigned long long)sh_cnt[i]);
      atomicAdd(&A.inst[inst].cnt[kLevels + l], sh_hsh[i]);
    }
  }
}

__global__ void trace_init_kernel(unsigned long long* ctl, unsigned long long n_roots) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl[CTL_HEAD] = 0;
    ctl[CTL_TAIL] = 0;
    ctl[CTL_OUTSTANDING] = n_roots;
    ctl[CTL_STATUS] = 0;
    ctl[CTL_EPOCH] = ctl[CTL_EPOCH] + 1;
  }
}

// Host-side launch helpers (called from api.cu).
cudaError_t launch_trace_init(unsigned long long* ctl, unsigned long long n_roots, cudaStream_t st) {
  trace_init_kernel<<<1, 32, 0, st>>>(ctl, n_roots);
  return cudaGetLastError();
}

cudaError_t trace_occupancy(int precision, int block, int* blocks_per_sm) {
  if (precision == RT_FP64)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_kernel<Walk64>, block, 0);
  return cudaErrorInvalidValue;
}

cudaError_t launch_trace(int precision, const TraceArgs& A, int grid, int block, cudaStream_t st) {
  if (precision == RT_FP64) {
    trace_kernel<Walk64><<<grid, block, 0, st>>>(A);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

}  // namespace rtg
