// policy.h -- host-side sizing and tuning rules of the library (plain C++,
// no CUDA), kept apart so they can be tested without a GPU.
#pragma once
#include <vector>

namespace rtg {

// Next attempt after a queue overflow of an automatically sized trace: grow
// the queue up to `limit` records, then split the sources into more passes.
// `peak` (records of the largest pass) undercounts the need, because dropped
// children were never expanded.  False when neither is possible.
inline bool grow_after_overflow(unsigned long long peak, unsigned long long limit, int nsrc, unsigned long long* cap,
                                int* passes) {
  if (*cap < limit) {
    const unsigned long long need = peak + peak / 4 + 1024;
    *cap = need > 4 * *cap ? need : 4 * *cap;
    if (*cap > limit) *cap = limit;
    return true;
  }
  if (*passes >= nsrc) return false;
  long long np = 2LL * *passes;
  const long long want = (long long)*passes * (long long)(peak / (limit / 2 + 1) + 1);
  if (want > np) np = want;
  if (np > nsrc) np = nsrc;
  *passes = (int)np;
  return true;
}

// Queue records a repeat of a trace can need at most: the three children of
// every split that went to other lanes (a split keeps child 0; which of the
// other three a free lane of the splitting warp takes instead of the queue
// depends on scheduling).  counts[l] = packages created at level l, four per
// split above level0.
template <class Count>
inline unsigned long long queue_worst_case(const Count* counts, int level0, int levels) {
  unsigned long long kids = 0;
  for (int l = level0 + 1; l < levels; ++l) kids += (unsigned long long)counts[l];
  return kids / 4 * 3;
}

// Segments a lane traces between visits to the queue, from the packages'
// mean length in the grid's last trace: long rays (optically thin media)
// gain from fewer warp-wide queue visits; without the in-warp hand-off of
// children (the finite-speed-of-light kernel) short ones gain from lanes
// that finish being refilled sooner.  Half the mean, as a power of two in
// [32, 64] with the hand-off (a lane whose package ends mostly takes a child
// that a split in its warp hands over, so short packages do not want short
// visits) and in [8, 64] without it; 16 before any trace was read back.
inline int tuned_segs_per_iter(double seg_per_pkg, bool handoff = true) {
  if (!(seg_per_pkg > 0)) return 16;
  int s = handoff ? 32 : 8;
  while (s < 64 && s < 0.5 * seg_per_pkg) s *= 2;
  return s;
}

// Halting radii of the next finite-speed-of-light trace (cell units): a
// package emitted a traces ago halts at neu[a]; neu[0] = c_dt and
// neu[a] = old[a - 1] + c_dt, the light travel summed since its emission.
// Ages whose previous radius lies beyond the box diagonal (+1 cell) cannot be
// in flight (a stored package is inside the box) and are dropped; `live`
// says whether the previous trace left packages in flight at all.
inline void flight_radii(const std::vector<double>& old, bool live, double c_dt, double diag,
                         std::vector<double>& neu) {
  size_t n_old = live ? old.size() : 0;
  while (n_old > 0 && old[n_old - 1] > diag + 1.0) --n_old;
  neu.assign(n_old + 1, 0.0);
  neu[0] = c_dt;
  for (size_t a = 1; a < neu.size(); ++a) neu[a] = old[a - 1] + c_dt;
}

}  // namespace rtg
